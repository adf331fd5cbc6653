// Batched execution of many independent contractions (the networks of many
// energy terms or graph instances): each stage of every contraction in a
// batch contributes its kernel jobs to shared job tables, and each table is
// launched once per stage.  Jobs keep the arithmetic of the single-call path
// (same plans, same tiles, same reduction orders), so a batched result is
// bit-identical to the one the same contraction gives alone.
//
// Job offsets are element offsets from one base pointer per kernel argument:
// a job built against its own buffers is rebased onto the lowest buffer of
// the launch (rounded down to 256 bytes, which keeps every buffer's
// alignment relative to the base, hence every vector-width and TMA
// alignment decision of the plan, valid).
#pragma once
#include <map>
#include <vector>

#include "tdplan.h"

namespace ftn {

// ---- collectors ------------------------------------------------------------------
struct PermBatch {
  struct Item {
    PermJob j;
    int64_t tiles;  // tiles of this job
    const char* src;
    char* dst;
  };
  std::vector<Item> items[2];  // [register-staged kernel, shared-memory-staged kernel]
  // Adds the finalised jobs of one plan table (tile_begin prefix sums over
  // total tiles) read from src and written to dst (hi plane).
  void add(const std::vector<PermJob>& jobs, int64_t total_tiles, int staged, const void* src, void* dst);
  bool empty() const { return items[0].empty() && items[1].empty(); }
};

// Launches both kernels of a PermBatch.  Split outputs write their lo plane
// at the hi address + lo_delta bytes (the same for every job).
ftn_status flush_perm(ftn_ctx ctx, PermBatch& pb, ftn_dtype in_type, int mode, int64_t lo_delta);

struct GemmF64Batch {
  struct Item {
    GemmProb g;  // offsets relative to a, b, c
    const double *a, *b;
    double* c;
  };
  struct RedItem {
    GemmProb r;  // a_off relative to part, c_off relative to c
    const double* part;
    double* c;
  };
  ftn_ctx ctx = nullptr;
  std::map<int, std::vector<Item>> by_bn;  // FP64 tile width -> problems
  std::vector<RedItem> red;                // split-K reductions (after the GEMMs)
  std::vector<void*> scratch;              // partial slabs, freed after the launches
  explicit GemmF64Batch(ftn_ctx c) : ctx(c) {}
  GemmF64Batch(const GemmF64Batch&) = delete;
  GemmF64Batch& operator=(const GemmF64Batch&) = delete;
  ~GemmF64Batch() {
    for (void* p : scratch) dev_free(ctx, p);
  }
};

// One problem set as a single-call launch would run it (tile width from the
// widest problem, FP64 split-K when the set has few tiles and is not split
// already); bounds are checked against the buffers' element counts.
ftn_status add_gemm_set(GemmF64Batch& gb, std::vector<GemmProb>& probs, const double* a, const double* b, double* c,
                        int64_t a_n, int64_t b_n, int64_t c_n);
// Adds already planned problems (tiles counted with bn) and their reductions.
void add_gemm_planned(GemmF64Batch& gb, const std::vector<GemmProb>& probs, int bn, const double* a, const double* b,
                      double* c);
void add_reductions(GemmF64Batch& gb, const std::vector<GemmProb>& red, const double* part, double* c);
// Launches the GEMMs (one launch per tile width), then the reductions.
ftn_status flush_gemm_f64(GemmF64Batch& gb);

// ---- small batched kernels (misc.cu) ------------------------------------------------
struct NormJob {
  void* x;
  int64_t n;
  double* logacc;
  unsigned long long* words;  // two max words (see normalize_tensor)
  int32_t cur;
  int32_t pad_;
  int64_t tile_begin;  // large jobs: first tile
};
// small: n <= 65536, one CTA each; large: max |x| and scale over tiles
ftn_status launch_normalize_batch(ftn_ctx ctx, ftn_dtype dt, const NormJob* d_small, int nsmall,
                                  const NormJob* d_large, int nlarge, int64_t large_tiles);
constexpr int64_t NORM_TILE = 8192;

struct CastJob {
  const void* src;
  void* dst;
  int64_t n;
  int64_t tile_begin;
};
constexpr int64_t CAST_TILE = 8192;
ftn_status launch_cast_batch(ftn_ctx ctx, ftn_dtype from, ftn_dtype to, const CastJob* d_jobs, int njobs,
                             int64_t tiles);

struct ResultJob {
  const void* value;  // rank-0 data, or null (no allowed entry: the value is 0)
  const double* logacc;
  int32_t f64;
  int32_t sign;  // the walk's sign (+1 or -1)
};
// out[2 i] = sign * value, out[2 i + 1] = log-scale accumulator
ftn_status launch_gather_results(ftn_ctx ctx, const ResultJob* d_jobs, int njobs, double* out);

// ---- batched operations ------------------------------------------------------------
struct TdItem {
  ftn_tensor A = nullptr, B = nullptr;
  int n = 0;
  int ax[MAXR] = {}, ay[MAXR] = {};
  uint64_t fa = 0, fb = 0;
  ftn_tensor C = nullptr;  // result (library-owned, created by the call)
};
// C = tensordot(A, B) for every item (no output permutation); all A and B
// share one dtype matching prec.
ftn_status tensordot_batch(ftn_ctx ctx, std::vector<TdItem>& items, ftn_prec prec);

struct CompressState;  // a compression's forward kept for its adjoint (compress.cu)

struct CompressItem {
  ftn_tensor X = nullptr, Y = nullptr;  // replaced by the compressed pair (inputs freed)
  int n = 0;
  int ax[MAXR] = {}, ay[MAXR] = {};
  int chi = 0;
  int arrows = 1;
  ftn_compress_info* info = nullptr;
  // ftn_compress_grad: cotangents of the compressed pair (tensors with the
  // new X's and Y's legs); when set, X and Y are left in place and dX, dY
  // receive the gradient with respect to them
  ftn_tensor gXn = nullptr, gYn = nullptr;
  ftn_tensor dX = nullptr, dY = nullptr;
  // keep X and Y (the caller still owns them) while X, Y are replaced by the
  // compressed pair
  bool keep_inputs = false;
  // a batch of one with keep_inputs: the forward's state (its workspace, job
  // and singular values) is kept in *keep_state for compress_backward, which
  // then runs the adjoint without recomputing the forward
  CompressState** keep_state = nullptr;
};
// ftn_compress for every item (FP64 tensors).
ftn_status compress_batch(ftn_ctx ctx, std::vector<CompressItem>& items);

// The adjoint of a kept compression (CompressItem::keep_state): gXn, gYn are
// the cotangents of the compressed pair, dX, dY receive new tensors with the
// inputs' legs.  The inputs must still be alive; the state stays valid (and
// is released by free_compress_state).
ftn_status compress_backward(ftn_ctx ctx, CompressState* st, ftn_tensor gXn, ftn_tensor gYn, ftn_tensor* dX,
                             ftn_tensor* dY);
void free_compress_state(CompressState* st);

struct NormItem {
  ftn_tensor t;
  void* d_state;  // [log accumulator, two max words]
  int step;
};
ftn_status normalize_batch(ftn_ctx ctx, const std::vector<NormItem>& items);

// out[i] = t[i] converted to dtype `to` (new library-owned tensors)
ftn_status cast_batch(ftn_ctx ctx, const std::vector<ftn_tensor>& t, ftn_dtype to, std::vector<ftn_tensor>& out);

}  // namespace ftn
