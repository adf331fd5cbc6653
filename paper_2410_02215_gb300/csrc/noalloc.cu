// ftn_tensordot_noalloc: the fermionic tensordot for callers that cannot
// allocate device memory themselves or through the library -- plug-in hosts
// that hand a library only the buffers they reserved up front, or processes
// whose device memory is owned by another framework's allocator and must not
// be grown behind its back.
//
// Everything the contraction needs beyond its inputs and output (the fused
// sector matrices, the plan tables, the device error word) is carved out of
// one file-scope static device array of FTN_NOALLOC_SCRATCH_BYTES.  Every
// GPU that loads this library holds that array until the process exits.
// Host code must never use the array's name as a device address: the name is
// a host-side stand-in.  The first call on each device (with that device
// current) asks the runtime for the array's device address once and caches
// it.  All calls share the array and it keeps the last call's contents (the
// error word at its start is cleared by every call).  Work of two calls that
// overlapped on the GPU would race on the array; this entry point prevents
// that by holding a host lock for the whole call and returning only after its
// work on the stream has finished (it synchronises the stream to read the
// error word, so a bounded wait that gave up is reported as FTN_ETIMEOUT).
#include <mutex>

#include "tdplan.h"

namespace ftn {
ftn_status tensordot_impl(ftn_ctx ctx, ftn_tensor A, ftn_tensor B, int n, const int* ax, const int* ay,
                          uint64_t flip_a, uint64_t flip_b, const int* out_perm, ftn_prec prec, ftn_tensor* C);
}

static __device__ __align__(256) unsigned char g_noalloc_scratch[FTN_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_noalloc_mu;
void* g_scratch_addr[256] = {};  // device address of the array, per device ordinal

struct Bump {
  unsigned char* base;
  size_t cap;
  size_t used;
};

// Sub-allocator over the static array for the duration of one call.
void* bump_alloc(size_t bytes, void* user) {
  Bump* b = static_cast<Bump*>(user);
  const size_t off = (b->used + 255) & ~(size_t)255;
  if (off > b->cap || bytes > b->cap - off) return nullptr;
  b->used = off + bytes;
  return b->base + off;
}
void bump_free(void*, void*) {}

}  // namespace

using namespace ftn;

extern "C" ftn_status ftn_tensordot_noalloc(void* cuda_stream, int rank_a, const int32_t* d_even_a,
                                            const int32_t* d_odd_a, const uint8_t* dual_a, int parity_a,
                                            const void* a, int rank_b, const int32_t* d_even_b,
                                            const int32_t* d_odd_b, const uint8_t* dual_b, int parity_b,
                                            const void* b, ftn_dtype dtype, int n, const int* axes_a,
                                            const int* axes_b, const int* out_perm, ftn_prec prec, void* c,
                                            int64_t c_capacity) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  int dev = 0;
  FTN_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return set_error(FTN_EINVAL, "device ordinal out of range");
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    FTN_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_addr[dev] = p;
  }
  Bump bump{static_cast<unsigned char*>(g_scratch_addr[dev]), FTN_NOALLOC_SCRATCH_BYTES, 0};
  ftn_ctx_s ctx;
  ctx.stream = (cudaStream_t)cuda_stream;
  ctx.alloc = bump_alloc;
  ctx.free_fn = bump_free;
  ctx.user = &bump;
  ctx.device = dev;
  ctx.tune = false;  // the tile-width tuner would take scratch per candidate and synchronise per run
  FTN_CUDA(cudaDeviceGetAttribute(&ctx.num_sms, cudaDevAttrMultiProcessorCount, dev));
  ctx.dev_err = (int*)bump_alloc(256, &bump);
  FTN_CUDA(cudaMemsetAsync(ctx.dev_err, 0, 256, ctx.stream));

  ftn_tensor A = nullptr, B = nullptr, C = nullptr;
  ftn_status st = ftn_tensor_wrap(&ctx, rank_a, d_even_a, d_odd_a, dual_a, parity_a, dtype, const_cast<void*>(a), &A);
  if (st == FTN_OK)
    st = ftn_tensor_wrap(&ctx, rank_b, d_even_b, d_odd_b, dual_b, parity_b, dtype, const_cast<void*>(b), &B);
  if (st == FTN_OK) st = validate_pairs(A, B, n, axes_a, axes_b);
  if (st == FTN_OK) {
    // result metadata: free legs of A then of B, optionally permuted
    const int cr = rank_a + rank_b - 2 * n;
    int32_t d0[MAXR], d1[MAXR];
    uint8_t du[MAXR];
    int k = 0;
    for (int i = 0; i < rank_a; ++i) {
      bool con = false;
      for (int j = 0; j < n; ++j) con = con || axes_a[j] == i;
      if (!con) d0[k] = d_even_a[i], d1[k] = d_odd_a[i], du[k] = dual_a[i], ++k;
    }
    for (int i = 0; i < rank_b; ++i) {
      bool con = false;
      for (int j = 0; j < n; ++j) con = con || axes_b[j] == i;
      if (!con) d0[k] = d_even_b[i], d1[k] = d_odd_b[i], du[k] = dual_b[i], ++k;
    }
    int32_t pd0[MAXR], pd1[MAXR];
    uint8_t pdu[MAXR];
    for (int u = 0; u < cr; ++u) {
      const int src = out_perm ? out_perm[u] : u;
      if (src < 0 || src >= cr) {
        st = set_error(FTN_EINVAL, "bad out_perm");
        break;
      }
      pd0[u] = d0[src], pd1[u] = d1[src], pdu[u] = du[src];
    }
    if (st == FTN_OK) st = ftn_tensor_wrap(&ctx, cr, pd0, pd1, pdu, parity_a ^ parity_b, dtype, c, &C);
    if (st == FTN_OK && C->numel > c_capacity)
      st = set_error(FTN_EINVAL, "ftn_tensordot_noalloc: output buffer holds fewer elements than the result");
  }
  if (st == FTN_OK) {
    st = tensordot_impl(&ctx, A, B, n, axes_a, axes_b, 0, 0, out_perm, prec, &C);
    if (st == FTN_ENOMEM)
      st = set_error(FTN_EINVAL,
                     "ftn_tensordot_noalloc: the contraction needs more scratch than the static "
                     "FTN_NOALLOC_SCRATCH_BYTES array provides");
  }
  if (st == FTN_OK) {
    // report a device-side bounded wait that gave up (error word at the array's start)
    int err = 0;
    cudaError_t e = cudaMemcpyAsync(&err, ctx.dev_err, sizeof(int), cudaMemcpyDeviceToHost, ctx.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx.stream);
    if (e != cudaSuccess)
      st = cuda_error(e, "ftn_tensordot_noalloc: reading the device error word");
    else if (err)
      st = set_error(FTN_ETIMEOUT, "ftn_tensordot_noalloc: a device-side bounded wait timed out");
  }
  clear_plan_caches(&ctx);  // releases plan tables into the (no-op) sub-allocator
  ftn_tensor_free(A);
  ftn_tensor_free(B);
  ftn_tensor_free(C);
  return st;
}
