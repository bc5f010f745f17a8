"""Failure detection without a GPU fault: the library's device-side waits are
bounded.  A wait on an mbarrier phase that nothing completes gives up after
its poll limit and reports PIC_ETIMEOUT through the C-ABI; the same wait
with its phase completed first succeeds; contexts before and after are
unaffected.  (No kernel here faults, traps or spins without a limit.)"""
import numpy as np
import pytest

from paper_1407_1810_gb300 import configs

from gpu_common import setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1407_1810_gb300 import build

    build.build()


def test_bounded_wait_reports_a_timeout_and_the_context_stays_usable():
    from paper_1407_1810_gb300 import picsar as P

    cfg = dict(configs.CONFIGS["monopole-64x64"], nr=16, nth=16, pairs_per_cell=2, precision="fp32")
    s, _, _, _ = setup(cfg)
    s.step(3)
    f0 = s.fields()
    for polls in (1, 1000):
        assert P.wait_selftest(polls, False) == P.PIC_ETIMEOUT
        assert b"gave up" in P.lib().pic_last_error()
        assert P.wait_selftest(polls, True) == P.PIC_OK
    assert P.wait_selftest(0, True) == P.PIC_EINVAL
    s.step(3)  # the context was not touched: it steps and reports no error
    assert s.moments()["step"] == 6
    assert np.all(np.isfinite(s.fields())) and not np.array_equal(s.fields(), f0)
