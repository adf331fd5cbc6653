// Internal declarations of libftn shared by the host runtime and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <map>
#include <mutex>
#include <unordered_map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/ftn.h"

namespace ftn {

constexpr int MAXR = FTN_MAX_RANK;

// Device-side error codes written into the context's error word.
constexpr int DEV_ERR_TIMEOUT = 1;

// ---- sign-permute job (one source block -> one destination layout) --------
// The source block is dense row-major.  Legs are split in three groups:
//   I: a suffix of the source legs (contiguous in the source, product PI),
//   O: legs with the smallest destination strides not in I (product PO),
//   B: the rest (product PB).
// A tile covers tr values of the O index times ti values of the I index for
// one batch index.  Two kernels share the job format: a shared-memory-staged
// one (16-byte cp.async copies of contiguous source rows into a
// shared-memory ring; needs 16-byte aligned rows) and a register-staged
// fallback with fixed 32 x 64 tiles.  finalize_perm_jobs() picks the kernel
// and the tiling.
constexpr int PERM_TI = 32;   // fallback tile: I extent
constexpr int PERM_GROUP_MIN = 32;   // I group (source-contiguous suffix): at least this many elements,
constexpr int PERM_GROUP_I = 128;    // grown further towards this many (never past PERM_GROUP_IMAX)
constexpr int PERM_GROUP_IMAX = 256;  // largest I grown beyond the minimum (whole in a tile for FP64 too)
constexpr int PERM_GROUP_O = 32;     // contiguous destination elements kept for the rows of a tile
constexpr int PERM_TO = 64;   // fallback tile: O extent
constexpr int PERM_TILE_BYTES = 16384;  // staged tile payload
constexpr int PERM_MAX_ROWS = 128;
constexpr int PERM_STAGES = 3;

struct PermJob {
  int64_t src_off;   // elements from the source base
  int64_t dst_off;   // elements from the destination base
  int64_t tile_begin;
  int64_t PB;
  int32_t PI, PO;
  int32_t tiles_i, tiles_o;
  int32_t nI, nO, nB;
  int32_t sign;      // +1 or -1
  int32_t store_fast_i;  // destination contiguous along the I index
  int32_t ti, tr;        // tile extents (I, O)
  int32_t bulk_ok;       // rows are 16-byte aligned with 16-byte multiple sizes
  int32_t vec4;          // quads along the store direction are contiguous and 4-element aligned
  int32_t iwrite;        // staged kernel: stores run along I in destination order (I whole in a tile)
  int32_t wmask;         // I legs (bit l = l-th I leg) forming the destination's contiguous run
  int32_t qw;            // elements of that run (product of the wmask legs)
  int32_t wsuf;          // the run is the innermost I legs in the same order: source columns run with it
  int32_t src_sel;       // source buffer: 0 = src, 1 = src1 (both operands of a contraction in one launch)
  int32_t dim[MAXR];     // I legs (source order), then O legs, then B legs
  int64_t sstr[MAXR];    // source strides
  int64_t dstr[MAXR];    // destination strides
};

// Output conversions of the sign-permute kernel.
enum PermMode {
  PERM_SAME = 0,      // same element type as the input
  PERM_TF32 = 1,      // FP32 -> TF32-rounded FP32
  PERM_TF32X2 = 2,    // FP32 -> TF32 hi + TF32 lo (two FP32 outputs)
  PERM_BF16 = 3,      // FP32 -> BF16
  PERM_BF16X2 = 4,    // FP32 -> BF16 hi + BF16 lo
  PERM_F16X2 = 5      // FP32 -> FP16 hi + FP16 lo
};

// Properties of the sector-GEMM precisions (see ftn_prec).
inline bool prec_valid(ftn_prec p) { return p >= FTN_PREC_F64 && p <= FTN_PREC_F16X3; }
inline bool prec_split(ftn_prec p) {
  return p == FTN_PREC_TF32X3 || p == FTN_PREC_BF16X3 || p == FTN_PREC_F16X3;
}
// 16-bit tensor-core operands (else TF32 in FP32 words, or FP64)
inline bool prec_half(ftn_prec p) { return p == FTN_PREC_BF16 || p == FTN_PREC_BF16X3 || p == FTN_PREC_F16X3; }
// the sign-permute's output conversion for the fused operand matrices
inline int prec_perm_mode(ftn_prec p) {
  switch (p) {
    case FTN_PREC_TF32: return PERM_TF32;
    case FTN_PREC_TF32X3: return PERM_TF32X2;
    case FTN_PREC_BF16: return PERM_BF16;
    case FTN_PREC_BF16X3: return PERM_BF16X2;
    case FTN_PREC_F16X3: return PERM_F16X2;
    default: return PERM_SAME;
  }
}

// ---- grouped sector GEMM problem: C[m, n] = sum_k A[m, k] B[n, k] ------------
// The result element (m, n) is stored at c_off + rowpart(m) + colpart(n)
// multiplied by c_sign, where rowpart/colpart expand m and n row-major over
// the row legs (rdim, rstr) and the column legs (cdim, cstr).  This places
// the result directly in a permuted output layout (the fermionic sign of the
// permutation is one sign per block).
struct GemmProb {
  int64_t tile_begin;
  int64_t a_off;   // element offset of the first A row (FP64 path)
  int64_t b_off;
  int64_t c_off;   // element offset of the output block
  int32_t M, N, K;
  int32_t pi;      // fused-matrix pair (bond parity sector)
  int32_t lda, ldb;
  int32_t a_row0, b_row0;  // first row inside the fused pi-matrices (TMA)
  int32_t tiles_m, tiles_n;
  int32_t c_sign;
  int32_t nrl, ncl;
  int32_t epi_rows;  // epilogue writes lane -> row (the destination is contiguous along rows)
  int32_t rdim[MAXR], cdim[MAXR];
  int64_t rstr[MAXR], cstr[MAXR];
  // FP64 path: element strides of the operands (A[m, k] = A[a_off + m*a_sm + k*a_sk])
  int64_t a_sm, a_sk, b_sn, b_sk;
  // FP64 path split-K: nsplit slices of kchunk, slice s written at c_off + s*c_slab
  int32_t nsplit, kchunk;
  int64_t c_slab;
  // tensor-core path tile order: problems sharing the same A rows (same pi
  // and row block) form a group whose tiles run m-tile by m-tile across all
  // its problems, so that concurrent CTAs reuse the A tile from L2.
  // tile_begin is the group's first tile for every member.
  int32_t grp_first, grp_count;
  int32_t row_tiles, tn_off;
  // 1: groups of 4 consecutive elements along the epilogue's write direction
  // are contiguous and 16-byte aligned in the destination (vector stores)
  int32_t vec4;
  // 1: the group's tiles run over its members' concatenated columns (their
  // column blocks are adjacent rows of B_pi and multiples of 32 wide); gcol
  // is this member's first column within the group
  int32_t gmerge;
  int32_t gcol;
  int32_t k0;  // tensor-core path: first K element of this problem (K-split parts)
};

// Offset of the row-major multi-index of x over n legs (last leg fastest),
// 32-bit index arithmetic (every leg dimension and every row or column
// index fits in 31 bits).
__host__ __device__ inline int64_t expand_index32(int x, int n, const int32_t* dim, const int64_t* str) {
  int64_t off = 0;
  for (int l = n - 1; l >= 0; --l) {
    const int d = dim[l];
    const int q = x / d;
    off += (int64_t)(x - q * d) * str[l];
    x = q;
  }
  return off;
}

// Same with 64-bit indices.
__host__ __device__ inline int64_t expand_index(int64_t x, int n, const int32_t* dim, const int64_t* str) {
  int64_t off = 0;
  for (int l = n - 1; l >= 0; --l) {
    const int64_t d = dim[l];
    const int64_t idx = x % d;
    x /= d;
    off += idx * str[l];
  }
  return off;
}

}  // namespace ftn

// ---- public opaque types -----------------------------------------------------
struct ftn_prof_rec {
  std::string label;
  cudaEvent_t a, b;
  double bytes, flops;
};

struct ftn_ctx_s {
  cudaStream_t stream = nullptr;
  ftn_alloc_fn alloc = nullptr;
  ftn_free_fn free_fn = nullptr;
  void* user = nullptr;
  int device = 0;
  int num_sms = 0;
  int* dev_err = nullptr;  // device error word (zeroed at creation)
  int64_t launches = 0;
  bool tune = true;  // tile-width tuning of large tensor-core plans (ftn_ctx_set_tuning)
  // grow-only workspace arena (reused by every call on this context)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // device blocks freed on this context, kept by size class for its later
  // allocations (dev_alloc / dev_free); block_class maps every live or cached
  // block to its class.  The lock covers frees from other host threads.
  std::mutex cache_mu;
  std::unordered_map<size_t, std::vector<void*>> free_blocks;
  std::unordered_map<void*, size_t> block_class;
  size_t cached_bytes = 0;
  // host buffer for the tables of batched launches (staging_begin)
  std::vector<uint8_t> stage;
  // pinned copies of the tables uploaded while the stream is captured into a
  // CUDA graph (the graph's copy nodes read them at every replay); freed with
  // the context
  std::vector<void*> graph_host;
  // per-launch profiling (ftn_ctx_profile)
  bool prof_on = false;
  std::vector<ftn_prof_rec> prof;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::string> prof_labels;
  std::string prof_tag;
};

struct ftn_tensor_s {
  ftn_ctx ctx = nullptr;
  int rank = 0;
  int32_t d0[FTN_MAX_RANK] = {};
  int32_t d1[FTN_MAX_RANK] = {};
  uint8_t dual[FTN_MAX_RANK] = {};
  int parity = 0;
  ftn_dtype dtype = FTN_F64;
  int64_t numel = 0;
  std::vector<int64_t> offsets;  // per block (index = mask >> 1)
  void* data = nullptr;
  bool owned = false;
};

namespace ftn {

// error handling (thread-local message)
ftn_status set_error(ftn_status st, const std::string& msg);
ftn_status cuda_error(cudaError_t e, const char* where);
#define FTN_CUDA(call)                                         \
  do {                                                         \
    cudaError_t _e = (call);                                   \
    if (_e != cudaSuccess) return ::ftn::cuda_error(_e, #call); \
  } while (0)
#define FTN_TRY(call)                      \
  do {                                     \
    ftn_status _s = (call);                \
    if (_s != FTN_OK) return _s;           \
  } while (0)

size_t dtype_size(ftn_dtype d);
void* dev_alloc(ftn_ctx ctx, size_t bytes);
void dev_free(ftn_ctx ctx, void* p);
// hands the context's cached free blocks back to the stream-ordered allocator
void release_cached_blocks(ftn_ctx ctx);
// Workspace of at least `bytes` (contents undefined), valid until the next
// call that asks for workspace on the same context.
void* workspace(ftn_ctx ctx, size_t bytes);
// Whether work on the stream is being captured into a CUDA graph.
bool stream_capturing(cudaStream_t s);
// The host source of a host-to-device copy: the buffer itself, or while the
// context's stream is captured, a pinned copy kept until the context goes
// (null if that allocation fails).
const void* capture_source(ftn_ctx ctx, const void* host, size_t bytes);

inline int popc(uint32_t x) { return __builtin_popcount(x); }
inline uint32_t block_mask(int rank, int parity, int64_t b) {
  if (rank == 0) return 0;
  uint32_t hi = (uint32_t)b << 1;
  return hi | (uint32_t)((popc(hi) + parity) & 1);
}
inline int64_t nblocks(int rank, int parity) {
  if (rank == 0) return parity == 0 ? 1 : 0;
  return (int64_t)1 << (rank - 1);
}
inline int64_t leg_dim(const ftn_tensor_s* t, int k, uint32_t mask) {
  return ((mask >> k) & 1) ? t->d1[k] : t->d0[k];
}
int64_t block_size(const ftn_tensor_s* t, uint32_t mask);

// creates a library-owned tensor with the given metadata
ftn_status make_tensor(ftn_ctx ctx, int rank, const int32_t* d0, const int32_t* d1, const uint8_t* dual,
                       int parity, ftn_dtype dtype, ftn_tensor* out);
bool same_meta(const ftn_tensor_s* a, int rank, const int32_t* d0, const int32_t* d1, const uint8_t* dual,
               int parity, ftn_dtype dtype);

// Permute-job builder: one source block (dims in source leg order, source
// contiguous row-major) to a destination with per-leg strides.
void add_perm_job(std::vector<PermJob>& jobs, int64_t& tiles, int rank, const int64_t* dims,
                  const int64_t* dst_strides, int64_t src_off, int64_t dst_off, int sign);

// Launch with programmatic stream serialisation: the kernel may begin while
// the kernel before it in the stream is still running.  Such a kernel only
// reads tables that no kernel writes before griddepcontrol.wait (pdl_wait),
// and signals griddepcontrol.launch_dependents only after that wait, so
// every grid earlier in the stream has completed by the time the next one
// can start.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t stream,
                       Args... args) {
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// kernel launchers (asynchronous on ctx->stream)
// Chooses the kernel (returns 1 for the shared-memory-staged one) and fills the tiling
// and tile prefix sums of every job; *tiles receives the total.
int finalize_perm_jobs(std::vector<PermJob>& jobs, size_t elem_size, int64_t* tiles, bool allow_staged);
ftn_status launch_permute(ftn_ctx ctx, const PermJob* d_jobs, int njobs, int64_t tiles, int staged, const void* src,
                          void* dst0, void* dst1, ftn_dtype in_type, int mode);
// The same with a second source buffer for the jobs with src_sel = 1.
ftn_status launch_permute2(ftn_ctx ctx, const PermJob* d_jobs, int njobs, int64_t tiles, int staged, const void* src,
                           const void* src1, void* dst0, void* dst1, ftn_dtype in_type, int mode);
// FP64 tiles are 64 x bn, bn in {16, 32, 64} (f64_pick_bn of the widest
// problem); the problems' tiles_n must be counted with the same bn.
ftn_status launch_gemm_f64(ftn_ctx ctx, const GemmProb* d_probs, int nprobs, int64_t tiles, const double* a,
                           const double* b, double* c, int bn);
int f64_pick_bn(int max_n);
// Small FP64 problems (at most F64W_MAX_MN outputs, at most F64W_MAX_K
// terms per output in their split slice) run on a warp kernel instead of the
// 64 x bn tiles: one warp per item of up to F64W_PASSES passes, each pass
// 32 / g outputs with g lanes splitting K (g from the problem's own K or
// split length only, so a problem's arithmetic never depends on the launch
// it is part of).  Longer dot products amortise a tile's overhead and reuse
// its operands from shared memory, so they stay on the tiled kernel.
struct WarpItem {
  int32_t prob;  // problem index in the launch's table
  int32_t ks;    // split-K slice
  int32_t e0;    // first output (row-major over M x N)
  int32_t cnt;   // outputs of this item
};
constexpr int64_t F64W_MAX_MN = 4096;
constexpr int F64W_MAX_K = 64;
constexpr int F64W_PASSES = 4;
inline bool f64w_small(const GemmProb& g) {
  return (int64_t)g.M * g.N <= F64W_MAX_MN && (g.nsplit > 1 ? g.kchunk : g.K) <= F64W_MAX_K;
}
// Tensor-core-precision problems go to the FP32 warp kernel only when, small
// as above, their dot products are also short (K <= TCW_MAX_K): a longer K
// amortises the tcgen05 tile's fixed cost even when the tile is mostly empty
// (32 x 32 sector blocks with K = 32 took 10 us on tcgen05 against 16.5 us on
// the warp kernel; the tiny, short-K problems of cluster networks gain from
// the warp kernel).
constexpr int TCW_MAX_K = 16;
inline bool tcw_small(const GemmProb& g) { return f64w_small(g) && g.K <= TCW_MAX_K; }
// K lanes: the largest power of two <= 32 that leaves each lane >= 8 terms
__host__ __device__ inline int f64w_klanes(int klen) {
  int g = 1;
  while (g < 32 && 16 * g <= klen) g *= 2;
  return g;
}
// appends the items of problem `prob` (all its split slices)
void f64w_items(const GemmProb& g, int prob, std::vector<WarpItem>& out);
ftn_status launch_gemm_f64_warp(ftn_ctx ctx, const GemmProb* d_probs, const WarpItem* d_items, int nitems,
                                const double* a, const double* b, double* c);
// The same for the tensor-core precisions' small problems: FP32 FMAs on the
// sum of the operand planes (lo plane lo_delta elements after the hi one).
ftn_status launch_gemm_f32_warp(ftn_ctx ctx, ftn_prec prec, const GemmProb* d_probs, const WarpItem* d_items,
                                int nitems, const void* a, const void* b, int64_t lo_delta, float* c);
// Partitions a planned FP64 problem list: tiled problems first (tile_begin
// recounted, returned tile total in tiles), the small ones after them with
// their items.  Returns the number of tiled problems.
int partition_f64(std::vector<GemmProb>& probs, std::vector<WarpItem>& items, int64_t& tiles);
// plain row-major output block (rows x cols, row stride ld) at c_off
void gemm_plain_output(GemmProb& g, int64_t c_off, int64_t ld);
// dst[e] = sum_s src[s * slab + e] for e < count (split-K reduction)
ftn_status launch_sum_slabs(ftn_ctx ctx, double* dst, const double* src, int64_t count, int nsplit, int64_t slab);
// FP64 split-K for launches with fewer than two tiles per SM: rewrites probs
// to write partial slabs (offsets into a separate buffer) and fills red with
// the reduction jobs carrying the original epilogues.  Returns the partial
// buffer's element count (0: no split, probs untouched); updates the tile
// count and sets red_total to the number of output elements.
int64_t plan_splitk_f64(std::vector<GemmProb>& probs, int num_sms, std::vector<GemmProb>& red, int64_t& tiles,
                        int64_t& red_total);
bool red_in_bounds(const std::vector<GemmProb>& red, int64_t part_n, int64_t c_n);
ftn_status launch_splitk_reduce(ftn_ctx ctx, const GemmProb* d_red, int nred, int64_t total, const double* part,
                                double* c);
// The same for FP32 partial slabs and output, added in FP64.
ftn_status launch_splitk_reduce_f32(ftn_ctx ctx, const GemmProb* d_red, int nred, int64_t total, const float* part,
                                    float* c);

// One tile of a tensor-core GEMM launch, decoded once when the plan is
// built: its problem (the group's first member when a tile spans a group's
// members), origin, bond sector, operand rows and K range.
struct TileEnt {
  int32_t prob, m0, n0, pi;
  int32_t a_y, b_y, K, k0;
};

struct TcOperands {
  // fused pi-matrices: rows x ldk elements, K-major; lo only for split modes
  const void* a_hi[2];
  const void* a_lo[2];
  const void* b_hi[2];
  const void* b_lo[2];
  int64_t a_rows[2], b_rows[2];
  int32_t kdim[2], ldk[2];
};
// tt: the launch's tile table (tc_tile_table), or null to decode tiles in the kernel.
ftn_status launch_gemm_tc(ftn_ctx ctx, ftn_prec prec, const TcOperands& ops, const GemmProb* d_probs, int nprobs,
                          int64_t tiles, int bn, float* c, const TileEnt* tt = nullptr);
// Fills d_out[t] for every tile t < tiles of a launch over d_probs (tile width bn).
ftn_status tc_tile_table(ftn_ctx ctx, const GemmProb* d_probs, int nprobs, int64_t tiles, int bn, TileEnt* d_out);
// Four TMA tensor maps (A hi, B hi, A lo, B lo) of one fused-matrix pair,
// encoded for tile width bn, as stored in a device table for batched launches.
struct alignas(64) TcMapSet {
  uint8_t bytes[4][128];
};
ftn_status tc_encode_set(ftn_prec prec, int bn, const TcOperands& ops, int pi, TcMapSet* out);
// Problem p reads its operands through d_maps[p.pi] (a device table, 64-byte aligned).
ftn_status launch_gemm_tc_maps(ftn_ctx ctx, ftn_prec prec, const TcMapSet* d_maps, const GemmProb* d_probs,
                               int nprobs, int64_t tiles, int bn, float* c);
int tc_pick_bn(int max_n, ftn_prec prec);
int64_t tc_tiles_for(int M, int N, int bn);

ftn_status upload_table(ftn_ctx ctx, const void* host, size_t bytes, void** dev);
// Table upload without an intermediate copy: staging_begin returns the
// context's host buffer (at least `bytes`, contents undefined) for the
// caller to fill; staging_upload copies its first `bytes` into a new device
// table on the context's stream.
void* staging_begin(ftn_ctx ctx, size_t bytes);
ftn_status staging_upload(ftn_ctx ctx, size_t bytes, void** dev);
// profiling brackets around one launch (no-ops unless profiling is enabled)
int prof_begin(ftn_ctx ctx, const char* label, double bytes, double flops);
void prof_end(ftn_ctx ctx, int rec);
void clear_plan_caches(ftn_ctx ctx);
// One kernel whose bounded mbarrier wait never completes (ftn_ctx_wait_selftest).
ftn_status launch_wait_selftest(ftn_ctx ctx, uint64_t limit_ns);
bool probs_in_bounds(const std::vector<GemmProb>& probs, int64_t a_n, int64_t b_n, int64_t c_n);

}  // namespace ftn
