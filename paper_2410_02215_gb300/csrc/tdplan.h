// Contraction plan shared by the tensordot and the compression code.
#pragma once
#include <string>
#include <unordered_map>

#include "common.h"

namespace ftn {

struct DevTables {
  ftn_ctx ctx;
  void* p = nullptr;
  ~DevTables() {
    if (p) dev_free(ctx, p);
  }
};

// Plan-cache key: the raw bytes of every field that determines a plan, in a
// fixed order, each variable-length part after its length (no text
// formatting: keys are built once per contraction step).
struct CacheKey {
  std::string s;
  CacheKey() { s.reserve(192); }
  template <typename T>
  CacheKey& put(T v) {
    s.append(reinterpret_cast<const char*>(&v), sizeof(T));
    return *this;
  }
  CacheKey& meta(const ftn_tensor_s* t) {
    put<int32_t>(t->rank).put<int32_t>(t->parity).put<int32_t>((int32_t)t->dtype);
    s.append(reinterpret_cast<const char*>(t->d0), sizeof(int32_t) * t->rank);
    s.append(reinterpret_cast<const char*>(t->d1), sizeof(int32_t) * t->rank);
    s.append(reinterpret_cast<const char*>(t->dual), t->rank);
    return *this;
  }
  CacheKey& ints(const int* v, int n) {
    put<int32_t>(n);
    for (int i = 0; i < n; ++i) put<int32_t>(v[i]);
    return *this;
  }
};

// ---------------------------------------------------------------------------------
struct TdPlan {
  int nfa = 0, nfb = 0, n = 0;
  int fa[MAXR], fb[MAXR];
  int64_t M[2] = {0, 0}, N[2] = {0, 0}, K[2] = {0, 0}, ldk[2] = {8, 8};
  int64_t afoff[2] = {0, 0}, bfoff[2] = {0, 0};
  int64_t af_elems = 0, bf_elems = 0;
  std::vector<PermJob> ja, jb, jc;
  int64_t ta = 0, tb = 0, tc = 0;
  int sa = 0, sb = 0, sc = 0;  // shared-memory-staged permute kernel usable
  // Both operands in one launch (B's jobs read the second source and write
  // after A's fused matrices): empty when the two need different kernels.
  std::vector<PermJob> jab;
  int64_t tab = 0;
  int sab = 0;
  bool fused = true;           // the GEMM epilogue writes the final layout
  std::vector<GemmProb> probs;
  int64_t gemm_tiles = 0;
  // FP64: probs[0, n_tiled) run on the tiled kernel, the rest (small
  // problems) on the warp kernel through witems
  int n_tiled = 0;
  std::vector<WarpItem> witems;
  // FP64 split-K (few output tiles): partial slabs and their reduction
  std::vector<GemmProb> red;
  int64_t part_elems = 0, red_total = 0;
  int bn = 0;
  bool out_perm = false;
  int cr = 0;  // result rank
  int32_t cd0[MAXR], cd1[MAXR];
  uint8_t cdual[MAXR];
  int cpar = 0;
  int64_t tmp_numel = 0;  // elements of the result
  // fused-matrix row/column offsets and sizes per pi, indexed by free-leg mask
  std::vector<int64_t> rowoff[2], rowsz[2], coloff[2], colsz[2];
  // device copies
  std::shared_ptr<DevTables> dev;
  PermJob* d_ja = nullptr;
  PermJob* d_jb = nullptr;
  PermJob* d_jc = nullptr;
  PermJob* d_jab = nullptr;
  TileEnt* d_tt = nullptr;  // tensor-core path: the decoded tiles of the GEMM launch
  bool tile_tab = false;
  GemmProb* d_probs = nullptr;
  GemmProb* d_red = nullptr;
  WarpItem* d_witems = nullptr;
};

// The cached plan of a contraction (built on first use; *fresh, when given,
// tells whether it was built by this call).
ftn_status get_plan(ftn_ctx ctx, const ftn_tensor_s* A, const ftn_tensor_s* B, int n, const int* ax, const int* ay,
                    uint64_t fa, uint64_t fb, const int* out_perm, ftn_prec prec, std::shared_ptr<TdPlan>& P,
                    bool* fresh = nullptr);
ftn_status validate_pairs(const ftn_tensor_s* A, const ftn_tensor_s* B, int n, const int* ax, const int* ay);
int inversion_parity(int r, const int* perm, uint32_t mask);
// bits legs[0..n) of mask, packed (bit i = bit legs[i])
uint32_t gather_bits(uint32_t mask, const int* legs, int n);
// masks over n legs with the given parity, in increasing order: offset and
// size of each (indexed by mask, -1 / 0 for the other parity) and the total
int64_t sector_offsets(int n, const int64_t* d0, const int64_t* d1, int parity, std::vector<int64_t>& off,
                       std::vector<int64_t>& size);
bool jobs_in_bounds(const std::vector<PermJob>& jobs, int64_t src_n, int64_t dst_n);
void clear_grad_caches(ftn_ctx ctx);
ftn_status tensordot_grad_impl(ftn_ctx ctx, ftn_tensor A, ftn_tensor B, ftn_tensor G, int n, const int* ax,
                               const int* ay, uint64_t flip_a, uint64_t flip_b, const int* out_perm, ftn_prec prec,
                               ftn_tensor* dA, ftn_tensor* dB);

}  // namespace ftn
