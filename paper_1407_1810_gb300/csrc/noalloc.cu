// noalloc.cu -- pic_get_particles_noalloc: export the live particles of a
// context into caller-owned device buffers without allocating device memory.
//
// Why: pic_get_particles allocates temporary device buffers and compacts the
// context.  Some callers cannot have the library call cudaMalloc: code that
// runs under a device-memory budget enforced by its own pool allocator, a
// host loop that cannot tolerate the implicit device synchronisation of an
// allocation, or a plugin that is handed pre-allocated device buffers and
// nothing else.  This entry point reads the context's particle slots as they
// are and writes the live ones (in slot order) into the caller's buffers.
//
// The only scratch memory is the file-scope array below: one 32-bit count per
// block of 256 particle slots plus a total, for at most PIC_NOALLOC_MAX_SLOTS
// slots.  Every GPU that loads the library holds it (4 MiB) until the process
// exits.  Its device address is looked up once per device by the first call on
// that device (make that first call outside any stream capture).  All calls
// share the array, so calls that overlap on the GPU (other streams, other
// threads) race on it; every call overwrites the counts it uses, so nothing
// has to be cleared between calls.
#include <mutex>
#include <string>

#include "pic_internal.h"

namespace {

constexpr int NB = 256;                                  // slots per block
constexpr int64_t MAX_SLOTS = (int64_t)1 << 28;          // PIC_NOALLOC_MAX_SLOTS
constexpr int64_t MAX_BLOCKS = MAX_SLOTS / NB;           // 2^20

static __device__ __align__(256) uint32_t g_block_counts[MAX_BLOCKS + 1];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
uint32_t *g_scratch[MAX_DEVICES] = {};

// device address of the scratch array on the current device (set-up once)
int scratch_ptr(uint32_t **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return pic_cuda_check(e, "cudaGetDevice");
  if (dev < 0 || dev >= MAX_DEVICES) return pic_fail(PIC_EINVAL, "device index beyond the no-alloc table");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_block_counts);
    if (e != cudaSuccess) return pic_cuda_check(e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_scratch[dev] = static_cast<uint32_t *>(p);
  }
  *out = g_scratch[dev];
  return PIC_OK;
}

template <typename Q>
__device__ inline bool live_slot(const Q *qw, int64_t k, int64_t n) {
  return k < n && qw[k] != Q(0);
}

template <typename Q>
__global__ void k_count_nc(const Q *__restrict__ qw, int64_t n, uint32_t *counts) {
  const int64_t k = blockIdx.x * (int64_t)NB + threadIdx.x;
  const int c = __syncthreads_count(live_slot(qw, k, n) ? 1 : 0);
  if (threadIdx.x == 0) counts[blockIdx.x] = (uint32_t)c;
}

// exclusive scan of nb counts in place by one block; counts[nb] = total
__global__ void k_scan_nc(uint32_t *counts, int64_t nb) {
  __shared__ uint32_t part[1024];
  const int t = threadIdx.x;
  const int64_t per = (nb + 1023) / 1024, b0 = t * per, b1 = min(nb, b0 + per);
  uint32_t s = 0;
  for (int64_t b = b0; b < b1; ++b) s += counts[b];
  part[t] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const uint32_t v = t >= off ? part[t - off] : 0u;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  uint32_t run = part[t] - s;
  for (int64_t b = b0; b < b1; ++b) {
    const uint32_t c = counts[b];
    counts[b] = run;
    run += c;
  }
  if (t == 1023) counts[nb] = part[1023];
}

struct Out {
  double *x1, *x2, *ur, *ut, *up, *qw;
  int64_t *id;
  int64_t cap;
};

__device__ inline int64_t out_slot(bool live, const uint32_t *offs) {
  __shared__ int wsum[NB / 32];
  const unsigned m = __ballot_sync(0xffffffffu, live);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) wsum[w] = __popc(m);
  __syncthreads();
  int base = 0;
  for (int q = 0; q < w; ++q) base += wsum[q];
  return (int64_t)offs[blockIdx.x] + base + __popc(m & ((1u << lane) - 1u));
}

__global__ void k_export_fp64_nc(pic::Parts64 P, int64_t n, const uint32_t *offs, Out O) {
  const int64_t k = blockIdx.x * (int64_t)NB + threadIdx.x;
  const bool live = live_slot(P.qw, k, n);
  const int64_t d = out_slot(live, offs);
  if (!live || d >= O.cap) return;
  O.x1[d] = P.x1[k]; O.x2[d] = P.x2[k];
  O.ur[d] = P.ur[k]; O.ut[d] = P.ut[k]; O.up[d] = P.up[k];
  O.qw[d] = P.qw[k];
  if (O.id) O.id[d] = P.id[k];
}

__global__ void k_export_fp32_nc(pic::Parts32 P, int64_t n, const uint32_t *offs, Out O) {
  const int64_t k = blockIdx.x * (int64_t)NB + threadIdx.x;
  const bool live = live_slot(P.qw, k, n);
  const int64_t d = out_slot(live, offs);
  if (!live || d >= O.cap) return;
  const uint32_t c = P.cell[k];
  O.x1[d] = (double)((int)(c >> 16) - pic::CELL_BIAS) + (double)P.dx[k];
  O.x2[d] = (double)(c & 0xffffu) + (double)P.dy[k];
  O.ur[d] = P.ur[k]; O.ut[d] = P.ut[k]; O.up[d] = P.up[k];
  O.qw[d] = P.qw[k];
  if (O.id) O.id[d] = P.id[k];
}

// A caller buffer must be memory of the context's device (or managed memory)
// before any kernel writes into it: a host pointer, or one of another GPU,
// would otherwise turn into an invalid device write instead of an error code.
int check_out(const pic_ctx *c, const void *p, const char *name) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the error the query left behind
    return pic_fail(PIC_EINVAL, std::string("pic_get_particles_noalloc: ") + name + " is not device memory");
  }
  const bool ok = a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == c->device);
  if (!ok)
    return pic_fail(PIC_EINVAL,
                    std::string("pic_get_particles_noalloc: ") + name + " is not memory of the context's device");
  return PIC_OK;
}

}  // namespace

extern "C" int pic_get_particles_noalloc(pic_ctx *c, int64_t *n, double *x1, double *x2, double *u_r,
                                         double *u_th, double *u_ph, double *qw, int64_t *id) {
  if (!c || !n) return pic_fail(PIC_EINVAL, "null argument");
  if (!x1 || !x2 || !u_r || !u_th || !u_ph || !qw) return pic_fail(PIC_EINVAL, "null output array");
  if (*n < 0) return pic_fail(PIC_EINVAL, "negative output capacity");
  {
    const void *bufs[7] = {x1, x2, u_r, u_th, u_ph, qw, id};
    const char *names[7] = {"x1", "x2", "u_r", "u_th", "u_ph", "qw", "id"};
    for (int k = 0; k < 7; ++k) {
      if (!bufs[k]) continue;  // only id may be NULL (checked above)
      const int e = check_out(c, bufs[k], names[k]);
      if (e) return e;
    }
  }
  const int64_t slots = c->n_used;
  if (slots > MAX_SLOTS)
    return pic_fail(PIC_EINVAL, "pic_get_particles_noalloc: the context holds more than 2^28 particle slots, "
                                "the size of the library's static scratch; use pic_get_particles");
  uint32_t *scratch = nullptr;
  int e = scratch_ptr(&scratch);
  if (e) return e;
  const int64_t nb = (slots + NB - 1) / NB;
  uint32_t total = 0;
  if (nb > 0) {
    const Out O{x1, x2, u_r, u_th, u_ph, qw, id, *n};
    if (c->d.precision == PIC_FP64) {
      k_count_nc<<<(unsigned)nb, NB, 0, c->stream>>>(c->p64.qw, slots, scratch);
      k_scan_nc<<<1, 1024, 0, c->stream>>>(scratch, nb);
      k_export_fp64_nc<<<(unsigned)nb, NB, 0, c->stream>>>(c->p64, slots, scratch, O);
    } else {
      k_count_nc<<<(unsigned)nb, NB, 0, c->stream>>>(c->p32.qw, slots, scratch);
      k_scan_nc<<<1, 1024, 0, c->stream>>>(scratch, nb);
      k_export_fp32_nc<<<(unsigned)nb, NB, 0, c->stream>>>(c->p32, slots, scratch, O);
    }
    PIC_CUDA(cudaGetLastError());
    PIC_CUDA(cudaMemcpyAsync(&total, scratch + nb, sizeof total, cudaMemcpyDeviceToHost, c->stream));
    PIC_CUDA(cudaStreamSynchronize(c->stream));
  }
  const int64_t cap = *n;
  *n = total;
  if ((int64_t)total > cap) return pic_fail(PIC_EINVAL, "output buffers too small (*n now holds the live count)");
  return pic_latch_status(c);  // errors latched by earlier steps, as every getter reports them
}
