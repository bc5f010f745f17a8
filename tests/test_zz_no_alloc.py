"""pic_get_particles_noalloc: the live-particle export for callers that must
not have the library allocate device memory (their own pool allocator, or a
host loop that cannot absorb an allocation's synchronisation).  Through the
C-ABI, on two calls in a row, its output must equal what pic_get_particles
returns for the same state (the same stored values, so exactly equal).
"""
import numpy as np
import pytest

from paper_1407_1810_gb300 import configs

from gpu_common import KEYS, by_id, setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1407_1810_gb300 import build

    build.build()


def _device_buffers(n):
    import torch

    out = {k: torch.empty(n, dtype=torch.float64, device="cuda") for k in KEYS}
    out["id"] = torch.empty(n, dtype=torch.int64, device="cuda")
    return out


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_export_matches_pic_get_particles(precision):
    # a hot plasma on a small grid: particles cross both conductors and are
    # deleted between the calls, so the context holds freed slots each time
    cfg = dict(configs.CONFIGS["monopole-64x64"], nr=24, nth=24, pairs_per_cell=3, T=1.0, precision=precision)
    import torch

    s, _, _, _ = setup(cfg, sort_interval=1000)
    for call in range(2):
        s.step(15)
        live = s.live()
        out = _device_buffers(live)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        n = s.particles_noalloc(out)
        free1 = torch.cuda.mem_get_info()[0]
        assert n == live
        if call == 1:  # after the first call's one-time symbol lookup: no device memory taken
            assert free1 == free0, (free0, free1)
        got = by_id({k: v[:n].cpu().numpy() for k, v in out.items()})
        ref = by_id(s.particles())  # the existing entry point (compacts the context)
        assert np.array_equal(got["id"], ref["id"]), call
        for k in KEYS:
            assert np.array_equal(got[k], ref[k]), (call, k)
        assert s.moments()["deleted"] > 0


def test_noalloc_reports_small_buffers():
    from paper_1407_1810_gb300 import picsar as P

    cfg = dict(configs.CONFIGS["monopole-64x64"], nr=16, nth=16, pairs_per_cell=2, precision="fp32")
    s, _, plasma, _ = setup(cfg)
    out = _device_buffers(10)
    with pytest.raises(P.PicError) as e:
        s.particles_noalloc(out)
    assert e.value.code == P.PIC_EINVAL


def test_noalloc_refuses_buffers_it_cannot_write():
    """A host array, a CPU tensor or a tensor of the wrong type is refused
    before any kernel runs (binding and C entry point)."""
    import ctypes

    import torch

    from paper_1407_1810_gb300 import picsar as P

    cfg = dict(configs.CONFIGS["monopole-64x64"], nr=16, nth=16, pairs_per_cell=2, precision="fp64")
    s, _, _, _ = setup(cfg)
    live = s.live()
    out = _device_buffers(live)
    for key, bad in (("x2", torch.empty(live, dtype=torch.float64)),
                     ("id", torch.empty(live, dtype=torch.int32, device="cuda")),
                     ("qw", torch.empty(2 * live, dtype=torch.float64, device="cuda")[::2])):
        with pytest.raises(ValueError):
            s.particles_noalloc(dict(out, **{key: bad}))
    host = np.empty(live)
    n = ctypes.c_int64(live)
    ptrs = [ctypes.c_void_p(out[k].data_ptr()) for k in KEYS]
    ptrs[3] = ctypes.c_void_p(host.ctypes.data)  # u_th on the host
    rc = P.lib().pic_get_particles_noalloc(s.h, ctypes.byref(n), *ptrs, None)
    assert rc == P.PIC_EINVAL
    assert b"u_th" in P.lib().pic_last_error()
    assert s.particles_noalloc(out) == live  # the context is unharmed
