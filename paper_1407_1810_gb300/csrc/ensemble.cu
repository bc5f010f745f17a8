// ensemble.cu -- an ensemble of independent simulations advanced together
// (batched launches in CUDA graphs) and the measurement-driven choice of the
// FP32 path's tile shape and sort interval, for one context or a whole
// ensemble.
#include <algorithm>
#include <array>
#include <chrono>
#include <cstring>
#include <vector>

#include "pic_internal.h"

using namespace pic;

// Ensemble with FP64 members: every member's steps up to the next sort of any
// member are captured, members on parallel branches (one forked stream each),
// into one CUDA graph that is launched once; the sorts run between graphs.  A
// captured graph is applied to the previous executable graph when its
// topology allows (cudaGraphExecUpdate), otherwise instantiated anew.
static int ensemble_branches(pic_ctx *const *ctxs, int n, int nsteps) {
  cudaStream_t origin;
  PIC_CUDA(cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking));
  std::vector<cudaStream_t> br(n);
  std::vector<cudaEvent_t> join(n);
  cudaEvent_t fork, after;
  PIC_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  PIC_CUDA(cudaEventCreateWithFlags(&after, cudaEventDisableTiming));
  for (int k = 0; k < n; ++k) {
    PIC_CUDA(cudaStreamCreateWithFlags(&br[k], cudaStreamNonBlocking));
    PIC_CUDA(cudaEventCreateWithFlags(&join[k], cudaEventDisableTiming));
  }
  // members' own streams finish their earlier work before the first graph
  for (int k = 0; k < n; ++k) PIC_CUDA(cudaStreamSynchronize(ctxs[k]->stream));
  cudaGraphExec_t exec = nullptr;
  int err = PIC_OK, done = 0;
  // A graph holds every member's steps up to the next sort of any member, so
  // each graph keeps all members on parallel branches; a member sorts only
  // when its own interval comes due.  (Letting each member's branch run to its
  // own next sort measured 13 % slower on the 64-member ensemble: the later
  // graphs hold fewer members.)
  while (done < nsteps && !err) {
    int block = nsteps - done;
    for (int k = 0; k < n; ++k) {
      pic_ctx *c = ctxs[k];
      block = std::min(block, std::max(1, c->d.sort_interval - c->steps_since_sort));
    }
    for (int k = 0; k < n && !err; ++k) {
      err = pic_prepare_steps(ctxs[k], block);
      if (!err) cudaStreamSynchronize(ctxs[k]->stream);
    }
    if (err) break;
    std::vector<cudaStream_t> own(n);
    std::vector<bool> prof(n);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) ce = cudaEventRecord(fork, origin);
    for (int k = 0; k < n && ce == cudaSuccess; ++k) {
      pic_ctx *c = ctxs[k];
      ce = cudaStreamWaitEvent(br[k], fork, 0);
      own[k] = c->stream;
      prof[k] = c->prof;
      c->stream = br[k];
      c->prof = false;
      for (int s = 0; s < block; ++s) pic_step_body(c);
      c->stream = own[k];
      c->prof = prof[k];
      if (ce == cudaSuccess) ce = cudaEventRecord(join[k], br[k]);
      if (ce == cudaSuccess) ce = cudaStreamWaitEvent(origin, join[k], 0);
    }
    cudaError_t ce2 = cudaStreamEndCapture(origin, &graph);
    if (ce == cudaSuccess) ce = ce2;
    if (ce == cudaSuccess) {
      bool fresh = exec == nullptr;
      if (!fresh) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(exec, graph, &info) != cudaSuccess) {
          cudaGetLastError();
          cudaGraphExecDestroy(exec);
          exec = nullptr;
          fresh = true;
        }
      }
      if (fresh) ce = cudaGraphInstantiate(&exec, graph, 0);
      if (ce == cudaSuccess) ce = cudaGraphLaunch(exec, origin);
      if (ce == cudaSuccess) ce = cudaEventRecord(after, origin);
    }
    if (graph) cudaGraphDestroy(graph);
    if (ce != cudaSuccess) { err = pic_cuda_check(ce, "ensemble graph"); break; }
    done += block;
    for (int k = 0; k < n && !err; ++k) {
      pic_ctx *c = ctxs[k];
      cudaStreamWaitEvent(c->stream, after, 0);
      if (c->steps_since_sort >= c->d.sort_interval) err = pic_compact(c);
    }
  }
  cudaStreamSynchronize(origin);
  if (exec) cudaGraphExecDestroy(exec);
  for (int k = 0; k < n; ++k) { cudaStreamDestroy(br[k]); cudaEventDestroy(join[k]); }
  cudaEventDestroy(fork);
  cudaEventDestroy(after);
  cudaStreamDestroy(origin);
  return err;
}

// ---- FP32 ensemble: one launch per phase for all members --------------------
// Each phase of a step is one kernel over the blocks of every member that
// takes part in it (a block finds its member by binary search over the
// launch's block offsets); the members' arguments for each step sit in a
// device table uploaded once per graph.  The kernels run the same per-block
// and per-node code as a single context's, so every member's result is
// bit-identical to its own pic_step run.  Steps up to the next sort of any
// member are captured into one CUDA graph; each member sorts when its own
// interval comes due.
namespace {

constexpr int ENS_MAX_BLOCK = 64;  // steps per graph at most

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Block maps of the grid phases: for each launch, every block's member and
// its block within that member ({member, block}); fixed for the call.
struct PhaseMaps {
  std::vector<std::vector<int2>> blk;
  explicit PhaseMaps(int nlists) : blk(nlists) {}
  void add(int list, int member, int blocks) {
    for (int b = 0; b < blocks; ++b) blk[list].push_back(make_int2(member, b));
  }
  int blocks(int list) const { return (int)blk[list].size(); }
};

// the tile kernel's member arguments (kernel parameters) of one step, per kind
struct StepTiles {
  std::vector<unsigned char> arg[ENS_TILE_KINDS];
  std::vector<int64_t> blocks[ENS_TILE_KINDS];
  void reset() {
    for (int q = 0; q < ENS_TILE_KINDS; ++q) { arg[q].clear(); blocks[q].clear(); }
  }
};

}  // namespace

static int ensemble_batched(pic_ctx *const *ctxs, int n, int nsteps, int64_t *kernels) {
  int max_filt = 0, max_smooth = 0;
  for (int k = 0; k < n; ++k) {
    max_filt = std::max(max_filt, ctxs[k]->d.n_filt);
    if (ctxs[k]->d.inject) max_smooth = std::max(max_smooth, ctxs[k]->d.inject_smooth);
  }
  // the grid phases in launch order, and which members take part in each
  const int L_FLUX = 0, L_FILT = L_FLUX + 1, L_NODES = L_FILT + max_filt, L_LOSSY = L_NODES + 1,
            L_GHOSTS = L_LOSSY + 1, L_COPY = L_GHOSTS + 1, L_SIGMA = L_COPY + 1, L_SMOOTH = L_SIGMA + 1,
            L_WRITE = L_SMOOTH + max_smooth, NLISTS = L_WRITE + 1;
  PhaseMaps maps(NLISTS);
  for (int k = 0; k < n; ++k) {
    const pic_ctx *c = ctxs[k];
    maps.add(L_FLUX, k, ens_blocks(c, ENS_FLUX));
    for (int p = 0; p < c->d.n_filt; ++p) maps.add(L_FILT + p, k, ens_blocks(c, ENS_FILTER));
    maps.add(L_NODES, k, ens_blocks(c, ENS_NODES));
    maps.add(L_LOSSY, k, ens_blocks(c, ENS_LOSSY));
    maps.add(L_GHOSTS, k, ens_blocks(c, ENS_GHOSTS));
    maps.add(L_COPY, k, ens_blocks(c, ENS_COPY32));
    if (c->d.inject) {
      maps.add(L_SIGMA, k, ens_blocks(c, ENS_SIGMA));
      for (int p = 0; p < c->d.inject_smooth; ++p) maps.add(L_SMOOTH + p, k, ens_blocks(c, ENS_SIGMA));
      maps.add(L_WRITE, k, ens_blocks(c, ENS_WRITE));
    }
  }
  std::vector<size_t> map_at(NLISTS + 1, 0);
  for (int q = 0; q < NLISTS; ++q) map_at[q + 1] = map_at[q] + maps.blk[q].size();
  const size_t tile_bytes = ens_tile_arg_bytes();
  const size_t step_sz = align_up((size_t)n * sizeof(EnsFieldArg), 256);
  unsigned char *h_tab = nullptr, *d_tab = nullptr;
  int2 *d_maps = nullptr;
  PIC_CUDA(cudaMallocHost((void **)&h_tab, step_sz * ENS_MAX_BLOCK));
  if (cudaMalloc((void **)&d_tab, step_sz * ENS_MAX_BLOCK) != cudaSuccess ||
      cudaMalloc((void **)&d_maps, std::max<size_t>(1, map_at[NLISTS]) * sizeof(int2)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(d_tab);
    cudaFreeHost(h_tab);
    return pic_fail(PIC_ENOMEM, "ensemble argument tables");
  }
  cudaStream_t origin = nullptr;
  cudaEvent_t after = nullptr;
  int err = PIC_OK;
  if (cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&after, cudaEventDisableTiming) != cudaSuccess)
    err = pic_fail(PIC_ECUDA, "ensemble stream");
  for (int q = 0; q < NLISTS && !err; ++q)
    if (!maps.blk[q].empty() &&
        cudaMemcpy(d_maps + map_at[q], maps.blk[q].data(), maps.blk[q].size() * sizeof(int2),
                   cudaMemcpyHostToDevice) != cudaSuccess)
      err = pic_fail(PIC_ECUDA, "ensemble block maps");
  for (int k = 0; k < n && !err; ++k) {
    cudaError_t ce = cudaStreamSynchronize(ctxs[k]->stream);  // earlier work of each member first
    if (ce != cudaSuccess) err = pic_cuda_check(ce, "ensemble member stream");
  }
  std::vector<StepTiles> tiles(ENS_MAX_BLOCK);
  std::vector<pic_ctx *> due;
  EnsSortScratch sort_scratch;
  cudaGraphExec_t exec = nullptr;
  int64_t launched = 0;
  int done = 0;
  while (done < nsteps && !err) {
    int block = std::min(nsteps - done, ENS_MAX_BLOCK);
    for (int k = 0; k < n; ++k) {
      pic_ctx *c = ctxs[k];
      block = std::min(block, std::max(1, c->d.sort_interval - c->steps_since_sort));
    }
    for (int k = 0; k < n && !err; ++k) {
      const int64_t l0 = ctxs[k]->launches;
      err = pic_prepare_steps(ctxs[k], block);
      launched += ctxs[k]->launches - l0;
      if (!err) cudaStreamSynchronize(ctxs[k]->stream);
    }
    if (err) break;
    // the members' arguments for each step; the host state advances as
    // step_body advances it (each member's launch count by the launches its
    // own step takes)
    for (int st = 0; st < block; ++st) {
      EnsFieldArg *fa = reinterpret_cast<EnsFieldArg *>(h_tab + (size_t)st * step_sz);
      StepTiles &T = tiles[st];
      T.reset();
      for (int k = 0; k < n; ++k) {
        pic_ctx *c = ctxs[k];
        const Grid &G = c->G;
        const int64_t tb = ens_tile_blocks(c);
        if (tb > 0) {
          const int kind = ens_tile_kind(c);
          std::vector<unsigned char> &ta = T.arg[kind];
          ta.resize(ta.size() + tile_bytes);
          ens_tile_arg(c, c->step * G.dt, ta.data() + ta.size() - tile_bytes);
          T.blocks[kind].push_back(tb);
          ++c->launches;
        }
        ens_fill_field_arg(c, &fa[k]);
        c->launches += 1 + 3 * (int64_t)c->d.n_filt + 3 + (ens_blocks(c, ENS_LOSSY) > 0) + 2;
        if (c->d.n_filt & 1)
          for (int q = 0; q < 3; ++q) std::swap(c->F[q], c->Ft[q]);
        c->step += 1;
        if (c->d.inject) {
          fa[k].t_inj = c->step * G.dt;
          fa[k].inj_base = c->n_used;
          fa[k].inj_id0 = c->next_id;
          fa[k].inj_step = (uint64_t)c->step;
          c->launches += 2 + c->d.inject_smooth;
          const int64_t nslots = (int64_t)G.nth * c->d.pairs_per_cell * 2;
          c->n_used += nslots;
          c->next_id += nslots;
        }
        c->steps_since_sort += 1;
      }
    }
    cudaError_t ce = cudaMemcpyAsync(d_tab, h_tab, step_sz * block, cudaMemcpyHostToDevice, origin);
    cudaGraph_t graph = nullptr;
    int64_t nodes = 0;
    if (ce == cudaSuccess) ce = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
      auto L = [&](int q) {
        EnsList x;
        x.blk = d_maps + map_at[q];
        return x;
      };
      for (int st = 0; st < block; ++st) {
        const EnsFieldArg *dfa = reinterpret_cast<const EnsFieldArg *>(d_tab + (size_t)st * step_sz);
        const StepTiles &T = tiles[st];
        for (int kind = 0; kind < ENS_TILE_KINDS; ++kind)
          if (!T.blocks[kind].empty())
            nodes += ens_tiles32(kind, T.arg[kind].data(), T.blocks[kind].data(), (int)T.blocks[kind].size(), origin);
        ens_flux_from_acc(dfa, L(L_FLUX), maps.blocks(L_FLUX), origin), ++nodes;
        for (int p = 0; p < max_filt; ++p)
          if (maps.blocks(L_FILT + p) > 0) ens_filter(dfa, L(L_FILT + p), maps.blocks(L_FILT + p), p, origin), ++nodes;
        ens_b_half(dfa, L(L_NODES), maps.blocks(L_NODES), origin);
        ens_e_full(dfa, L(L_NODES), maps.blocks(L_NODES), origin);
        ens_b_half(dfa, L(L_NODES), maps.blocks(L_NODES), origin);
        nodes += 3;
        if (maps.blocks(L_LOSSY) > 0) ens_lossy(dfa, L(L_LOSSY), maps.blocks(L_LOSSY), origin), ++nodes;
        ens_ghosts(dfa, L(L_GHOSTS), maps.blocks(L_GHOSTS), origin);
        ens_copy32(dfa, L(L_COPY), maps.blocks(L_COPY), origin);
        nodes += 2;
        if (maps.blocks(L_SIGMA) > 0) {
          ens_inject_sigma(dfa, L(L_SIGMA), maps.blocks(L_SIGMA), origin), ++nodes;
          for (int p = 0; p < max_smooth; ++p)
            if (maps.blocks(L_SMOOTH + p) > 0)
              ens_inject_smooth(dfa, L(L_SMOOTH + p), maps.blocks(L_SMOOTH + p), p, origin), ++nodes;
          ens_inject_write(dfa, L(L_WRITE), maps.blocks(L_WRITE), origin), ++nodes;
        }
      }
      cudaError_t ce2 = cudaStreamEndCapture(origin, &graph);
      if (ce == cudaSuccess) ce = ce2;
    }
    if (ce == cudaSuccess) {
      bool fresh = exec == nullptr;
      if (!fresh) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(exec, graph, &info) != cudaSuccess) {
          cudaGetLastError();
          cudaGraphExecDestroy(exec);
          exec = nullptr;
          fresh = true;
        }
      }
      if (fresh) ce = cudaGraphInstantiate(&exec, graph, 0);
      if (ce == cudaSuccess) ce = cudaGraphLaunch(exec, origin);
      if (ce == cudaSuccess) ce = cudaEventRecord(after, origin);
    }
    if (graph) cudaGraphDestroy(graph);
    if (ce != cudaSuccess) { err = pic_cuda_check(ce, "ensemble graph"); break; }
    launched += nodes;
    done += block;
    // the members whose sort is due, sorted together after the graph
    due.clear();
    for (int k = 0; k < n; ++k) {
      pic_ctx *c = ctxs[k];
      cudaStreamWaitEvent(c->stream, after, 0);
      if (c->steps_since_sort >= c->d.sort_interval) due.push_back(c);
    }
    if (!due.empty()) {
      int64_t nk = 0;
      err = ens_sort32(due.data(), (int)due.size(), origin, sort_scratch, &nk);
      launched += nk;
    }
    // the staging table is refilled next: its copy must have completed
    if (!err) cudaEventSynchronize(after);
  }
  if (origin) cudaStreamSynchronize(origin);
  if (exec) cudaGraphExecDestroy(exec);
  if (after) cudaEventDestroy(after);
  if (origin) cudaStreamDestroy(origin);
  ens_sort_scratch_free(sort_scratch);
  cudaFree(d_maps);
  cudaFree(d_tab);
  cudaFreeHost(h_tab);
  if (kernels) *kernels = launched;
  return err;
}

extern "C" int pic_ensemble_step(pic_ctx *const *ctxs, int32_t n, int32_t nsteps, int64_t *kernels) {
  if (!ctxs || n <= 0 || nsteps < 0) return pic_fail(PIC_EINVAL, "bad ensemble arguments");
  for (int k = 0; k < n; ++k)
    if (!ctxs[k]) return pic_fail(PIC_EINVAL, "null ensemble member");
  const int dev = ctxs[0]->device;
  bool fp32 = true;
  for (int k = 0; k < n; ++k) {
    if (ctxs[k]->device != dev) return pic_fail(PIC_EINVAL, "ensemble members on different devices");
    fp32 = fp32 && ctxs[k]->d.precision == PIC_FP32;
  }
  for (int k = 0; k < n; ++k)
    for (int q = 0; q < k; ++q)
      if (ctxs[q] == ctxs[k]) return pic_fail(PIC_EINVAL, "a context appears twice in the ensemble");
  int err;
  if (fp32) {
    err = ensemble_batched(ctxs, n, nsteps, kernels);
  } else {
    int64_t l0 = 0;
    for (int k = 0; k < n; ++k) l0 += ctxs[k]->launches;
    err = ensemble_branches(ctxs, n, nsteps);
    if (kernels) {
      int64_t l1 = 0;
      for (int k = 0; k < n; ++k) l1 += ctxs[k]->launches;
      *kernels = l1 - l0;
    }
  }
  if (err) return err;
  for (int k = 0; k < n; ++k) {
    const int e = pic_latch_status(ctxs[k]);
    if (e) return e;
  }
  return PIC_OK;
}

extern "C" int pic_autotune(pic_ctx *c, int32_t trial_steps, int32_t *sort_interval, int32_t *tile_shape) {
  if (!c || trial_steps < 1) return pic_fail(PIC_EINVAL, "bad autotune arguments");
  if (c->d.precision != PIC_FP32) return pic_fail(PIC_EINVAL, "autotune applies to the FP32 path");
  const int shapes[3] = {0, 1, 2}, intervals[4] = {5, 10, 20, 40};
  double best = 1e300;
  int best_shape = c->d.tile_shape, best_s = c->d.sort_interval;
  cudaEvent_t e0, e1;
  PIC_CUDA(cudaEventCreate(&e0));
  PIC_CUDA(cudaEventCreate(&e1));
  int err = PIC_OK;
  for (int sh : shapes) {
    for (int S : intervals) {
      pic_ctx *k = nullptr;
      if ((err = pic_clone_context(c, &k))) break;
      k->d.sort_interval = S;
      if (sh != k->d.tile_shape) err = pic_set_tiles(k, sh);
      if (!err) err = pic_step(k, S);  // warm-up: one full sort cycle
      const int n = std::max(trial_steps, 2 * S);
      if (!err) {
        cudaEventRecord(e0, k->stream);
        err = pic_step(k, n);
        cudaEventRecord(e1, k->stream);
        cudaEventSynchronize(e1);
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      pic_destroy(k);
      if (err) break;
      if (ms / n < best) { best = ms / n; best_shape = sh; best_s = S; }
    }
    if (err) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err) return err;
  c->d.sort_interval = best_s;
  if (best_shape != c->d.tile_shape && (err = pic_set_tiles(c, best_shape))) return err;
  if (sort_interval) *sort_interval = best_s;
  if (tile_shape) *tile_shape = best_shape;
  return PIC_OK;
}

// One tile shape and sort interval for every member of an ensemble, by
// measurement of the batched step itself: each candidate runs on clones of all
// members through pic_ensemble_step, timed on the host clock (the batched
// step's cost includes its host work), and the fastest is applied to every
// member.  A shape and an interval shared by all members keep each step's tile
// launches and sorts to one batch each.
extern "C" int pic_autotune_ensemble(pic_ctx *const *ctxs, int32_t n, int32_t trial_steps, int32_t *sort_interval,
                                     int32_t *tile_shape) {
  if (!ctxs || n <= 0 || trial_steps < 1) return pic_fail(PIC_EINVAL, "bad autotune arguments");
  for (int k = 0; k < n; ++k) {
    if (!ctxs[k]) return pic_fail(PIC_EINVAL, "null ensemble member");
    if (ctxs[k]->d.precision != PIC_FP32) return pic_fail(PIC_EINVAL, "autotune applies to the FP32 path");
    for (int q = 0; q < k; ++q)
      if (ctxs[q] == ctxs[k]) return pic_fail(PIC_EINVAL, "a context appears twice in the ensemble");
  }
  const int shapes[3] = {0, 1, 2}, intervals[3] = {10, 20, 40};
  double best = 1e300;
  int best_shape = ctxs[0]->d.tile_shape, best_s = ctxs[0]->d.sort_interval;
  int err = PIC_OK;
  std::vector<pic_ctx *> cl(n, nullptr);
  for (int sh : shapes) {
    for (int S : intervals) {
      for (int k = 0; k < n && !err; ++k) {
        err = pic_clone_context(ctxs[k], &cl[k]);
        if (!err) {
          cl[k]->d.sort_interval = S;
          if (sh != cl[k]->d.tile_shape) err = pic_set_tiles(cl[k], sh);
        }
      }
      if (!err) err = pic_ensemble_step(cl.data(), n, S, nullptr);  // warm-up: one full sort cycle
      const int m = std::max(trial_steps, 2 * S);
      double ms = 0.0;
      if (!err) {
        const auto t0 = std::chrono::steady_clock::now();
        err = pic_ensemble_step(cl.data(), n, m, nullptr);
        ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      }
      for (int k = 0; k < n; ++k) {
        pic_destroy(cl[k]);
        cl[k] = nullptr;
      }
      if (err) break;
      if (ms / m < best) { best = ms / m; best_shape = sh; best_s = S; }
    }
    if (err) break;
  }
  if (err) return err;
  for (int k = 0; k < n; ++k) {
    pic_ctx *c = ctxs[k];
    c->d.sort_interval = best_s;
    if (best_shape != c->d.tile_shape && (err = pic_set_tiles(c, best_shape))) return err;
  }
  if (sort_interval) *sort_interval = best_s;
  if (tile_shape) *tile_shape = best_shape;
  return PIC_OK;
}

