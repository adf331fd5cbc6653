// Bond compression ftn_compress (Sec. II.A: symmetric QR/SVD with the chi
// largest singular values pooled over all symmetry blocks; Sec. II.B: the
// decomposition runs after transposing into row | column order).
//
// GPU pipeline, FP64 throughout, per bond-parity sector pi:
//   1. sign-permute X -> X_pi = [free_X | bond] and Y -> Y_pi^T = [free_Y | bond]
//      (the fused layouts of the tensordot, bond parity of the arrow folded in);
//   2. R factors of X_pi and Y_pi^T by Householder QR (only R is formed):
//      each CTA streams a chunk of rows through shared memory into its own
//      triangular factor, and a binary tree of the same kernel merges the
//      chunks' factors (TSQR); a side with no more rows than bond states
//      uses the matrix itself (X_pi = I * X_pi);
//   3. core M_pi = R_X R_Y^T and its SVD by one-sided (Hestenes) Jacobi;
//   4. one host synchronisation: the singular values of both sectors are
//      pooled and the chi largest kept;
//   5. X' = X_pi (R_Y^T V_k S_k^{-1/2}) and Y'^T = Y_pi^T (R_X^T U_k S_k^{-1/2}),
//      written straight into the block layouts of the new tensors.
// Step 5 is the projector form of X' = Q_X U sqrt(S), Y' = sqrt(S) V^T Q_Y^T:
// Q_X U_k S_k = X R_Y^T V_k, so no orthogonal factor is ever formed.  With
// chi at or above the rank, op(X', Y') = op(X, Y) exactly for any invertible
// R factors; below it the truncation is that of the exact SVD as long as the
// R factors are backward stable (Householder: R^T R = (X + E)^T (X + E) with
// |E| ~ eps |X|, whatever the condition of X).
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>

#include "batch.h"
#include "ptx.cuh"

namespace ftn {

constexpr int LA_THREADS = 512;
constexpr int LA_MAX_DIM = 1024;  // largest bond sector handled by the Jacobi SVD

// One pass of the streaming Householder QR: the rows of src (rows x K, row
// stride ld) are appended to the upper-triangular factor R (K x K row-major,
// global memory) and R is updated so that R_new^T R_new = R^T R + src^T src.
struct QrJob {
  const double* src;
  double* R;
  int64_t rows, ld;
  int K;
  int init;  // 0: R starts as zero; 1: R holds a factor to extend
  int tri;   // 1: src is upper triangular (row i is zero before column i)
};

struct SvdJob {
  const double* T;  // n x m row-major input, left untouched
  double* Tf;       // n x m output: the rows orthogonalised (row j = s_j u_j^T)
  double* s;        // n singular values (row norms at convergence)
  int* sweeps;      // sweeps used (diagnostic)
  int n, m;
};

// Cluster Jacobi: SVDC_WARPS warps per CTA (one per SM sub-partition), rows
// of up to 32 * SVDC_MAX_E elements held in registers while a pair is
// rotated, and at most SVDC_SMEM_BYTES of rows per CTA.
constexpr int SVDC_WARPS = 4;
constexpr int SVDC_MAX_E = 16;
constexpr int SVDC_SMEM_BYTES = 192 * 1024;

struct GatherJob {
  const double* left;   // source row (length nl)
  const double* right;  // source row (length nr)
  double* dl;
  double* dr;
  double sl, sr;  // scale factors
  int nl, nr;
  double* dsc;    // receives sc (the norm the n-side vector of this state gets)
  double sc;
};

// Kept n-side singular vectors of one bond sector: k rows of length n (row
// stride n) in decreasing singular value, row j scaled to norm sc[j].
struct OrthJob {
  double* v;
  const double* sc;
  int k, n;
};

constexpr int QR_ROWS = 16;      // rows of src per pass (one per lane of warp 0 in the norm)
constexpr int QR_THREADS = 128;

// Householder QR, R factor only (Sec. II.A: the QR of each symmetry block).
// Rows arrive in blocks of QR_ROWS held in shared memory.  For column j with
// x = [a; b] = [R_jj; B(:, j)] the reflector H = I - tau v v^T, v = [1; b / (a
// - beta)], beta = -sign(a) |x|, tau = (beta - a) / beta in [1, 2], maps x to
// [beta; 0] and is applied to the trailing columns of R row j and of the
// block (the form of LAPACK's dlarfg: |x| is taken after scaling by max|x|,
// and no intermediate can overflow, however small b has become).  Row j of R
// is read and written only at step j, so R stays in global memory (it is
// L2-resident and each access is one coalesced row).  A column whose block
// part is zero, or below 2^-960 in magnitude, needs no reflector (this also
// skips the zero prefix of triangular sources).  Once a short block's rank
// is absorbed its rows hold only rounding noise, which every further group
// of reflectors shrinks by ~2^-52: that is where such tiny columns arise.
__global__ void __launch_bounds__(QR_THREADS) qr_stream_kernel(const QrJob* jobs) {
  extern __shared__ double qb[];  // QR_ROWS x K, row-major
  __shared__ double refl[2];      // tau, 1 / (a - beta)
  __shared__ int skip;
  const QrJob J = jobs[blockIdx.x];
  const int K = J.K, t = threadIdx.x, lane = t & 31, warp = t >> 5;
  double* R = J.R;
  if (!J.init)
    for (int64_t e = t; e < (int64_t)K * K; e += blockDim.x) R[e] = 0.0;
  for (int64_t r0 = 0; r0 < J.rows; r0 += QR_ROWS) {
    const int nb = (int)(J.rows - r0 < QR_ROWS ? J.rows - r0 : QR_ROWS);
    __syncthreads();  // the previous block's last column is done (and R is zeroed)
    for (int e = t; e < QR_ROWS * K; e += blockDim.x) {
      const int i = e / K, c = e - i * K;
      qb[e] = i < nb ? J.src[(r0 + i) * J.ld + c] : 0.0;
    }
    __syncthreads();
    const int j0 = J.tri ? (int)(r0 < K ? r0 : K) : 0;
    for (int j = j0; j < K; ++j) {
      if (warp == 0) {
        const double bj = lane < QR_ROWS ? qb[lane * K + j] : 0.0;
        double mx = fabs(bj);
        for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        int sk = 1;
        if (mx > 0x1p-960) {
          const double a = R[(int64_t)j * K + j];
          const double sc = fmax(mx, fabs(a));
          const double u = bj / sc;
          double ss = u * u;
          for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
          if (lane == 0) {
            const double as = a / sc;
            const double nrm = sc * sqrt(fma(as, as, ss));
            const double beta = a > 0.0 ? -nrm : nrm;
            refl[0] = (beta - a) / beta;
            refl[1] = 1.0 / (a - beta);
            R[(int64_t)j * K + j] = beta;
          }
          sk = 0;
        }
        if (lane == 0) skip = sk;
      }
      __syncthreads();
      if (!skip) {
        const double tau = refl[0], id = refl[1];
        for (int c = j + 1 + t; c < K; c += blockDim.x) {
          double* rp = R + (int64_t)j * K + c;
          const double rjc = *rp;
          double w = 0.0;
#pragma unroll
          for (int i = 0; i < QR_ROWS; ++i) w = fma(qb[i * K + j], qb[i * K + c], w);
          w = tau * fma(w, id, rjc);
          *rp = rjc - w;
          const double wv = w * id;
#pragma unroll
          for (int i = 0; i < QR_ROWS; ++i) qb[i * K + c] = fma(-wv, qb[i * K + j], qb[i * K + c]);
        }
      }
      __syncthreads();
    }
  }
}

// Sum of three per-lane values over the warp with 6 additions instead of 15:
// the first two levels split the lanes between the values.  Every lane gets
// the three totals.
__device__ __forceinline__ void warp_sum3(double& a, double& b, double& c) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const bool h16 = lane & 16, h8 = lane & 8;
  double k = h16 ? b : a;
  k += __shfl_xor_sync(full, h16 ? a : b, 16);
  c += __shfl_xor_sync(full, c, 16);
  double k2 = h8 ? c : k;
  k2 += __shfl_xor_sync(full, h8 ? k : c, 8);
  k2 += __shfl_xor_sync(full, k2, 4);
  k2 += __shfl_xor_sync(full, k2, 2);
  k2 += __shfl_xor_sync(full, k2, 1);
  a = __shfl_sync(full, k2, 0);
  b = __shfl_sync(full, k2, 16);
  c = __shfl_sync(full, k2, 8);
}

// Jacobi rotation for the pair (t_p, t_q) with al = |t_p|^2, be = |t_q|^2,
// ga = t_p . t_q: returns false when the pair is orthogonal to the
// tolerance (|ga| <= tol |t_p| |t_q|).  The tangent of the rotation angle,
// t = 2 ga sgn(d) / (|d| + sqrt(d^2 + 4 ga^2)) with d = be - al, is formed in
// FP32 from the pair scaled by a power of two; c = (1 + t^2)^{-1/2} and
// s = c t are then formed in FP64 from that t, so the rotation is orthogonal
// to FP64 rounding whatever the accuracy of the angle (an angle off by a
// relative 1e-7 leaves 1e-7 of ga, removed in the next sweep).
__device__ __forceinline__ bool jacobi_rotation(double al, double be, double ga, double tol2, double& c,
                                                double& s) {
  if (!(ga * ga > tol2 * (al * be))) return false;
  const double d = be - al, g2 = 2.0 * ga;
  const double h = fmax(fabs(d), fabs(g2));
  const int e = (__double2hiint(h) >> 20) & 0x7ff;
  if (e == 0 || e >= 2046) return false;  // subnormal or non-finite pair: leave it
  const double sc = __hiloint2double((2046 - e) << 20, 0);  // 2^(1023 - e): h * sc in [1, 2)
  const float df = (float)(d * sc), gf = (float)(g2 * sc);
  const float tf = copysignf(1.0f, df) * gf / (fabsf(df) + sqrtf(df * df + gf * gf));
  const double t = (double)tf;
  c = rsqrt(fma(t, t, 1.0));
  s = c * t;
  return true;
}

// One-sided (Hestenes) Jacobi: orthogonalise the n rows of an n x m matrix
// T by plane rotations in round-robin order (n/2 disjoint pairs per round).
// Converged when a sweep applies no rotation, i.e. every pair satisfies
// |t_p . t_q| <= m eps |t_p| |t_q| (a computed dot product of length m
// carries rounding of about m eps relative to |t_p| |t_q|, so a tighter test
// would never be met).  Then T_f = Q^T T has rows s_j u_j^T (u_j the right
// singular vectors of T) and the left ones follow as q_j = T u_j / s_j
// (re-orthogonalised for the kept states, orth_rows_kernel), so the rotations
// themselves are never accumulated.
__device__ __forceinline__ double jacobi_tol2(int m) {
  const double tol = (double)(m > 8 ? m : 8) * 2.220446049250313e-16;
  return tol * tol;
}

// Rows whose squared norm is at or below tau2 = (m eps |T|_F)^2 are
// numerically zero: rounding in a rotation with a row of norm |T| moves them
// by about their own size, so they are never rotated, they leave the
// round-robin at the next sweep boundary, and their singular value is
// reported as exactly 0.  (A rank-deficient core would otherwise keep its
// rounding-level rows rotating until the sweep limit.)
__device__ __forceinline__ double jacobi_tau2(int m, double fro2) {
  const double f = (double)(m > 8 ? m : 8) * 2.220446049250313e-16;
  return f * f * fro2;
}

__device__ __forceinline__ void round_robin_pair(int k, int r, int np, int& p, int& q) {
  const int a = k, b = np - 1 - k;
  p = a == 0 ? 0 : 1 + (a - 1 + r) % (np - 1);
  q = b == 0 ? 0 : 1 + (b - 1 + r) % (np - 1);
}

// Single-CTA version over a matrix in global memory (rows longer than the
// cluster kernel holds in registers).
__device__ __forceinline__ void jacobi_rows(double* A, int n, int m, int* rotated, double* s_out, int* sweeps_out,
                                            double tau2) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int np = n + (n & 1);
  const double tol2 = jacobi_tol2(m);
  int sweep = 0;
  for (; sweep < 40 && np > 1; ++sweep) {
    if (threadIdx.x == 0) *rotated = 0;
    __syncthreads();
    for (int r = 0; r < np - 1; ++r) {
      for (int k = warp; k < np / 2; k += nw) {
        int p, q;
        round_robin_pair(k, r, np, p, q);
        if (p >= n || q >= n) continue;
        double* ap = A + (int64_t)p * m;
        double* aq = A + (int64_t)q * m;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int i = lane; i < m; i += 32) {
          const double x = ap[i], y = aq[i];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        warp_sum3(al, be, ga);
        if (al <= tau2 || be <= tau2) continue;
        double c, sn;
        if (!jacobi_rotation(al, be, ga, tol2, c, sn)) continue;
        for (int i = lane; i < m; i += 32) {
          const double x = ap[i], y = aq[i];
          ap[i] = fma(c, x, -sn * y);
          aq[i] = fma(sn, x, c * y);
        }
        if (lane == 0) *rotated = 1;
      }
      __syncthreads();
    }
    if (!*rotated) break;
    __syncthreads();
  }
  if (threadIdx.x == 0) *sweeps_out = sweep;
  for (int j = warp; j < n; j += nw) {
    double ss = 0.0;
    for (int i = lane; i < m; i += 32) ss = fma(A[(int64_t)j * m + i], A[(int64_t)j * m + i], ss);
    for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (lane == 0) s_out[j] = ss > tau2 ? sqrt(ss) : 0.0;
  }
}

__global__ void __launch_bounds__(LA_THREADS) svd_rows_global_kernel(const SvdJob* jobs) {
  __shared__ int rotated;
  __shared__ double red[33];
  const SvdJob jb = jobs[blockIdx.x];
  const int64_t nm = (int64_t)jb.n * jb.m;
  double ss = 0.0;
  for (int64_t e = threadIdx.x; e < nm; e += blockDim.x) {
    const double v = jb.T[e];
    jb.Tf[e] = v;
    ss = fma(v, v, ss);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if (lane == 0) red[warp] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    red[32] = t;
  }
  __syncthreads();
  jacobi_rows(jb.Tf, jb.n, jb.m, &rotated, jb.s, jb.sweeps, jacobi_tau2(jb.m, red[32]));
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t map_rank(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ double ld_cluster(uint32_t a) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void st_cluster(uint32_t a, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}
__device__ __forceinline__ int ld_cluster_s32(uint32_t a) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}
// Hardware barrier over all threads of the cluster; release/acquire makes the
// shared-memory writes of every CTA visible to all of them.
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

__device__ __forceinline__ unsigned ld_cluster_u8(uint32_t a) {
  unsigned short v;
  asm volatile("ld.shared::cluster.u8 %0, [%1];" : "=h"(v) : "r"(a) : "memory");
  return v;
}

// Cluster Jacobi: one cluster of C CTAs per matrix.  Row i lives in the
// shared memory of CTA i mod C (slot i / C); each round the C * SVDC_WARPS
// warps take the round's pairs of live rows, read both rows through
// distributed shared memory into registers, and write the rotated rows back
// in place; a cluster barrier separates the rounds.  Spreading a matrix over
// C SMs multiplies the FP64 rate the rotations get by C.  The list of live
// rows is rebuilt identically in every CTA at each sweep boundary.
template <int E>
__global__ void __launch_bounds__(SVDC_WARPS * 32) svd_rows_cluster_kernel(const SvdJob* jobs, int C) {
  extern __shared__ __align__(16) double rows[];
  __shared__ int flag[2];
  __shared__ double part;
  __shared__ int act[LA_MAX_DIM];
  __shared__ unsigned char live[LA_MAX_DIM];  // this CTA's slots
  __shared__ unsigned char all_live[LA_MAX_DIM];
  __shared__ int n_act;
  __shared__ double rnorm[LA_MAX_DIM];  // this CTA's squared row norms
  const uint32_t rank = cluster_rank();
  const SvdJob jb = jobs[blockIdx.x / C];
  const int n = jb.n, m = jb.m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nloc = ((int)(n - rank) + C - 1) / C;  // rows rank, rank + C, ...
  for (int l = 0; l < nloc; ++l)
    for (int i = threadIdx.x; i < m; i += blockDim.x) rows[(int64_t)l * m + i] = jb.T[(int64_t)(l * C + rank) * m + i];
  if (threadIdx.x == 0) flag[0] = flag[1] = 0;
  __syncthreads();
  // squared row norms (one warp per row, lanes strided along the row)
  for (int l = warp; l < nloc; l += SVDC_WARPS) {
    const double* r = rows + (int64_t)l * m;
    double q = 0.0;
    for (int i = lane; i < m; i += 32) q = fma(r[i], r[i], q);
    for (int o = 16; o; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if (lane == 0) rnorm[l] = q;
  }
  const uint32_t base = smem_u32(rows);
  cluster_sync_all();
  // |T|_F^2 as the sum of the row norms in row order (lane-strided, then the
  // shuffle tree): the same arithmetic for every cluster size, so a matrix's
  // decomposition does not depend on the C it is launched with
  if (warp == 0) {
    double q = 0.0;
    for (int i = lane; i < n; i += 32) {
      double v;
      asm volatile("ld.shared::cluster.f64 %0, [%1];"
                   : "=d"(v)
                   : "r"(map_rank(smem_u32(&rnorm[i / C]), (uint32_t)(i % C)))
                   : "memory");
      q += v;
    }
    for (int o = 16; o; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if (lane == 0) part = q;
  }
  __syncthreads();
  const double fro2 = part;
  const double tol2 = jacobi_tol2(m), tau2 = jacobi_tau2(m, fro2);

  // marks this CTA's live rows, then (after a cluster barrier) rebuilds the
  // ordered list of live rows from all CTAs' marks
  auto mark_live = [&]() {
    for (int l = warp; l < nloc; l += SVDC_WARPS) {
      const double* r = rows + (int64_t)l * m;
      double q = 0.0;
      for (int i = lane; i < m; i += 32) q = fma(r[i], r[i], q);
      for (int o = 16; o; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
      if (lane == 0) live[l] = q > tau2 ? 1 : 0;
    }
  };
  auto build_list = [&]() {
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      all_live[i] = (unsigned char)ld_cluster_u8(map_rank(smem_u32(&live[i / C]), (uint32_t)(i % C)));
    __syncthreads();
    if (warp == 0) {
      int run = 0;
      for (int b0 = 0; b0 < n; b0 += 32) {
        const int i = b0 + lane;
        const bool on = i < n && all_live[i];
        const unsigned bal = __ballot_sync(0xffffffffu, on);
        if (on) act[run + __popc(bal & ((1u << lane) - 1u))] = i;
        run += __popc(bal);
      }
      if (lane == 0) n_act = run;
    }
    __syncthreads();
  };
  mark_live();
  cluster_sync_all();
  build_list();

  const int gw = (int)rank * SVDC_WARPS + warp, nwarps = C * SVDC_WARPS;
  int sweep = 0;
  for (; sweep < 40; ++sweep) {
    const int na = n_act;
    const int np = na + (na & 1);
    for (int r = 0; r + 1 < np; ++r) {
      for (int k = gw; k < np / 2; k += nwarps) {
        int pa, qa;
        round_robin_pair(k, r, np, pa, qa);
        if (pa >= na || qa >= na) continue;
        const int p = act[pa], q = act[qa];
        const uint32_t ap = map_rank(base + (uint32_t)((p / C) * m) * 8u, (uint32_t)(p % C));
        const uint32_t aq = map_rank(base + (uint32_t)((q / C) * m) * 8u, (uint32_t)(q % C));
        double x[E], y[E];
        double al = 0.0, be = 0.0, ga = 0.0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int i = lane + 32 * e;
          x[e] = i < m ? ld_cluster(ap + 8u * i) : 0.0;
          y[e] = i < m ? ld_cluster(aq + 8u * i) : 0.0;
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
          al = fma(x[e], x[e], al);
          be = fma(y[e], y[e], be);
          ga = fma(x[e], y[e], ga);
        }
        warp_sum3(al, be, ga);
        if (al <= tau2 || be <= tau2) continue;
        double c, sn;
        if (!jacobi_rotation(al, be, ga, tol2, c, sn)) continue;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int i = lane + 32 * e;
          if (i < m) {
            st_cluster(ap + 8u * i, fma(c, x[e], -sn * y[e]));
            st_cluster(aq + 8u * i, fma(sn, x[e], c * y[e]));
          }
        }
        if (lane == 0) flag[sweep & 1] = 1;
      }
      cluster_sync_all();
      // every CTA read the other flag at the end of the previous sweep,
      // before this barrier: clear it for the next sweep
      if (r == 0 && threadIdx.x == 0) flag[(sweep + 1) & 1] = 0;
    }
    const int any = lane < C ? ld_cluster_s32(map_rank(smem_u32(&flag[sweep & 1]), (uint32_t)lane)) : 0;
    if (!__any_sync(0xffffffffu, any != 0)) break;
    // peers finished reading the marks before the first barrier of this sweep
    mark_live();
    cluster_sync_all();
    build_list();
  }
  if (rank == 0 && threadIdx.x == 0) *jb.sweeps = sweep;
  for (int l = warp; l < nloc; l += SVDC_WARPS) {
    const double* src = rows + (int64_t)l * m;
    double* dst = jb.Tf + (int64_t)(l * C + rank) * m;
    double q = 0.0;
    for (int i = lane; i < m; i += 32) {
      const double v = src[i];
      q = fma(v, v, q);
      dst[i] = v;
    }
    for (int o = 16; o; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if (lane == 0) jb.s[l * C + rank] = q > tau2 ? sqrt(q) : 0.0;
  }
  cluster_sync_all();  // no CTA leaves while a peer may still read its flags
}

struct CompactJob {
  const double* src;  // rows x cols, leading dimension ld
  double* dst;        // the nonzero rows, packed (leading dimension cols)
  int* count;         // number of nonzero rows
  int rows, cols, ld;
};

// Packs the rows of an R factor that are not identically zero (rows of
// dropped Cholesky pivots, or zero rows of a short matrix used as its own
// factor).  They add nothing to M = R_X R_Y^T, so leaving them out gives the
// same nonzero singular triplets from a smaller core.  rows <= LA_MAX_DIM.
__global__ void __launch_bounds__(256) compact_rows_kernel(const CompactJob* jobs) {
  __shared__ unsigned char nz[LA_MAX_DIM];
  __shared__ int chunk_off[LA_MAX_DIM / 32 + 1];
  const CompactJob jb = jobs[blockIdx.x];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = warp; r < jb.rows; r += nw) {
    bool any = false;
    for (int c = lane; c < jb.cols; c += 32) any |= jb.src[(int64_t)r * jb.ld + c] != 0.0;
    any = __any_sync(0xffffffffu, any);
    if (lane == 0) nz[r] = any ? 1 : 0;
  }
  __syncthreads();
  const int nchunk = (jb.rows + 31) / 32;
  if (warp == 0) {
    int run = 0;
    for (int ch = 0; ch < nchunk; ++ch) {
      const int r = ch * 32 + lane;
      const unsigned b = __ballot_sync(0xffffffffu, r < jb.rows && nz[r]);
      if (lane == 0) chunk_off[ch] = run;
      run += __popc(b);
    }
    if (lane == 0) {
      chunk_off[nchunk] = run;
      *jb.count = run;
    }
  }
  __syncthreads();
  for (int r = warp; r < jb.rows; r += nw) {
    if (!nz[r]) continue;
    const int ch = r / 32;
    int pos = chunk_off[ch];
    for (int q = ch * 32; q < r; ++q) pos += nz[q];
    for (int c = lane; c < jb.cols; c += 32) jb.dst[(int64_t)pos * jb.cols + c] = jb.src[(int64_t)r * jb.ld + c];
  }
}

__global__ void gather_kernel(const GatherJob* jobs) {
  const GatherJob g = jobs[blockIdx.x];
  for (int i = threadIdx.x; i < g.nl; i += blockDim.x) g.dl[i] = g.left[i] * g.sl;
  for (int i = threadIdx.x; i < g.nr; i += blockDim.x) g.dr[i] = g.right[i] * g.sr;
  if (threadIdx.x == 0) *g.dsc = g.sc;
}

// The n-side vector q_j = T u_j / s_j inherits from u_j its rounding
// components along the other singular directions, multiplied by s_i / s_j:
// about m eps s_max / s_j along the directions of larger singular values,
// which the projector form would amplify by s_j^{-1}.  Classical Gram-Schmidt
// applied twice against the kept vectors of larger singular value (already
// cleaned, in decreasing order) removes those components; the result keeps
// both residuals |T u_j - s_j q_j| and |T^T q_j - s_j u_j| at the rounding
// level of T, which is what the projectors X R_Y^T V S^{-1/2} need.  Rows
// are renormalised to their target norms sc[j] = s_j^{-1/2}.
__global__ void __launch_bounds__(256) orth_rows_kernel(const OrthJob* jobs) {
  __shared__ double h[LA_MAX_DIM];
  __shared__ double red[9];
  const OrthJob J = jobs[blockIdx.x];
  const int n = J.n, t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < J.k; ++j) {
    double* vj = J.v + (int64_t)j * n;
    for (int pass = 0; pass < 2 && j > 0; ++pass) {
      for (int i = warp; i < j; i += nw) {
        const double* vi = J.v + (int64_t)i * n;
        double d = 0.0;
        for (int e = lane; e < n; e += 32) d = fma(vi[e], vj[e], d);
        for (int o = 16; o; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) h[i] = d / (J.sc[i] * J.sc[i]);
      }
      __syncthreads();
      for (int e = t; e < n; e += blockDim.x) {
        double a = vj[e];
        for (int i = 0; i < j; ++i) a = fma(-h[i], J.v[(int64_t)i * n + e], a);
        vj[e] = a;
      }
      __syncthreads();
    }
    double q = 0.0;
    for (int e = t; e < n; e += blockDim.x) q = fma(vj[e], vj[e], q);
    for (int o = 16; o; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if (lane == 0) red[warp] = q;
    __syncthreads();
    if (t == 0) {
      double tot = 0.0;
      for (int w = 0; w < nw; ++w) tot += red[w];
      red[8] = tot > 0.0 ? J.sc[j] / sqrt(tot) : 0.0;
    }
    __syncthreads();
    const double f = red[8];
    for (int e = t; e < n; e += blockDim.x) vj[e] *= f;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------
namespace {

template <typename T>
ftn_status put_table(ftn_ctx ctx, const std::vector<T>& v, void** d) {
  return upload_table(ctx, v.data(), v.size() * sizeof(T), d);
}

struct DevBuf {
  ftn_ctx ctx;
  void* p = nullptr;
  explicit DevBuf(ftn_ctx c) : ctx(c) {}
  ~DevBuf() {
    if (p) dev_free(ctx, p);
  }
};

GemmProb make_prob(int M, int N, int K, int64_t a_off, int64_t a_sm, int64_t a_sk, int64_t b_off, int64_t b_sn,
                   int64_t b_sk) {
  GemmProb g;
  std::memset(&g, 0, sizeof(g));
  g.M = M;
  g.N = N;
  g.K = K;
  g.a_off = a_off;
  g.a_sm = a_sm;
  g.a_sk = a_sk;
  g.b_off = b_off;
  g.b_sn = b_sn;
  g.b_sk = b_sk;
  g.tiles_m = (M + 63) / 64;
  g.tiles_n = (N + 63) / 64;
  return g;
}

template <int E>
ftn_status setup_svd_cluster(int* cmax) {
  auto k = svd_rows_cluster_kernel<E>;
  FTN_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SVDC_SMEM_BYTES));
  FTN_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  if (E == 1) {  // probe once whether 16-CTA clusters with full shared memory can be resident
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(SVDC_WARPS * 32);
    cfg.dynamicSmemBytes = SVDC_SMEM_BYTES;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 16;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int num = 0;
    if (cudaOccupancyMaxActiveClusters(&num, k, &cfg) != cudaSuccess) {
      (void)cudaGetLastError();
      num = 0;
    }
    *cmax = num >= 1 ? 16 : 8;
  }
  return FTN_OK;
}

// Largest cluster size the Jacobi kernel uses on this device (16 where
// non-portable clusters of that size fit, else the portable 8).
int svd_cluster_max(ftn_ctx ctx) {
  static std::mutex mu;
  static int cmax[64] = {0};
  const int dev = ctx->device >= 0 && ctx->device < 64 ? ctx->device : 0;
  std::lock_guard<std::mutex> lock(mu);
  if (!cmax[dev]) {
    int c = 8;
    if (setup_svd_cluster<1>(&c) != FTN_OK || setup_svd_cluster<2>(&c) != FTN_OK ||
        setup_svd_cluster<4>(&c) != FTN_OK || setup_svd_cluster<8>(&c) != FTN_OK ||
        setup_svd_cluster<16>(&c) != FTN_OK)
      c = 8;
    cmax[dev] = c;
  }
  return cmax[dev];
}

template <int E>
ftn_status launch_svd_cluster_e(ftn_ctx ctx, const SvdJob* jobs, int njobs, int C, size_t smem) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(C * njobs));
  cfg.blockDim = dim3(SVDC_WARPS * 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  FTN_CUDA(cudaLaunchKernelEx(&cfg, svd_rows_cluster_kernel<E>, jobs, C));
  ctx->launches += 1;
  return FTN_OK;
}

ftn_status launch_svd_cluster(ftn_ctx ctx, const SvdJob* jobs, int njobs, int C, int E, size_t smem) {
  switch (E) {
    case 1: return launch_svd_cluster_e<1>(ctx, jobs, njobs, C, smem);
    case 2: return launch_svd_cluster_e<2>(ctx, jobs, njobs, C, smem);
    case 4: return launch_svd_cluster_e<4>(ctx, jobs, njobs, C, smem);
    case 8: return launch_svd_cluster_e<8>(ctx, jobs, njobs, C, smem);
    case 16: return launch_svd_cluster_e<16>(ctx, jobs, njobs, C, smem);
    default: return set_error(FTN_EINVAL, "internal error: Jacobi row length");
  }
}

}  // namespace

namespace {

// Per-job state of a batched compression (one bond of one pair of tensors).
// Offsets are in doubles from the job's own workspace.
struct CJob {
  CompressItem* it = nullptr;
  std::shared_ptr<TdPlan> P;
  int64_t ws_n = 0, ws_off = 0;
  double* ws = nullptr;
  int64_t o_xf = 0, o_yf = 0;
  int64_t o_gx[2], o_gy[2], o_m[2], o_tf[2], o_wk[2], o_zk[2], o_px[2], o_qy[2], o_ms3[2], o_rxc[2], o_ryc[2],
      o_sc[2];
  int64_t s_off[2];  // singular values + sweep count in the batch's shared buffer
  // Householder TSQR of the tall sides: chunks of qr_lx / qr_ly rows, one
  // K x K factor slot per chunk at o_gx / o_gy (slot 0 holds the result)
  int64_t qr_lx[2], qr_ly[2];
  int qr_px[2], qr_py[2];
  int rx[2], ry[2], ldx[2], ldy[2], nrot[2], mlen[2];
  int64_t rx_off[2], ry_off[2];
  bool tall_x[2], tall_y[2], trans[2];
  struct Cand {
    double s;
    int pi, idx;
  };
  std::vector<Cand> kept;  // kept singular values, largest first
  int k[2] = {0, 0};
  ftn_tensor Xn = nullptr, Yn = nullptr;
};

ftn_status cj_prepare(ftn_ctx ctx, CJob& J) {
  CompressItem& it = *J.it;
  ftn_tensor X = it.X, Y = it.Y;
  if (!X || !Y) return set_error(FTN_EINVAL, "null argument");
  if (X->dtype != FTN_F64 || Y->dtype != FTN_F64)
    return set_error(FTN_EUNSUPPORTED, "ftn_compress works on FP64 tensors");
  if (it.chi < 0) return set_error(FTN_EINVAL, "chi must be >= 0");
  if (it.n < 1) return set_error(FTN_EINVAL, "a bond needs at least one leg pair");
  FTN_TRY(validate_pairs(X, Y, it.n, it.ax, it.ay));
  uint64_t flip = 0;
  if (!it.arrows)  // cancel the arrow parity: plain ordered contraction F(XY)
    for (int i = 0; i < it.n; ++i)
      if (X->dual[it.ax[i]] == 0) flip |= 1ull << it.ax[i];
  FTN_TRY(get_plan(ctx, X, Y, it.n, it.ax, it.ay, flip, 0, nullptr, FTN_PREC_F64, J.P));
  const TdPlan* P = J.P.get();
  for (int pi = 0; pi < 2; ++pi)
    if (P->K[pi] > LA_MAX_DIM) return set_error(FTN_EUNSUPPORTED, "bond sector larger than the batched Jacobi SVD handles");
  // ---- workspace layout (doubles) ----
  auto al = [](int64_t x) { return (x + 31) / 32 * 32; };
  int64_t off = 0;
  J.o_xf = off;
  off += al(P->af_elems);
  J.o_yf = off;
  off += al(P->bf_elems);
  for (int pi = 0; pi < 2; ++pi) {
    const int64_t K = P->K[pi], R = P->M[pi], Cc = P->N[pi];
    J.tall_x[pi] = R > K;
    J.tall_y[pi] = Cc > K;
    J.rx[pi] = (int)std::min(R, K);
    J.ry[pi] = (int)std::min(Cc, K);
    // chunks of at least 2K rows (the merge tree then adds at most ~1/6 of
    // the leaves' work), at most 256 per side
    auto chunk_rows = [&](int64_t rows) {
      int64_t L = std::max<int64_t>({2 * K, (rows + 255) / 256, (int64_t)QR_ROWS});
      return (L + QR_ROWS - 1) / QR_ROWS * QR_ROWS;
    };
    J.qr_lx[pi] = J.tall_x[pi] ? chunk_rows(R) : 0;
    J.qr_px[pi] = J.tall_x[pi] ? (int)((R + J.qr_lx[pi] - 1) / J.qr_lx[pi]) : 0;
    J.qr_ly[pi] = J.tall_y[pi] ? chunk_rows(Cc) : 0;
    J.qr_py[pi] = J.tall_y[pi] ? (int)((Cc + J.qr_ly[pi] - 1) / J.qr_ly[pi]) : 0;
    J.o_gx[pi] = off;
    off += al((int64_t)J.qr_px[pi] * K * K);
    J.o_gy[pi] = off;
    off += al((int64_t)J.qr_py[pi] * K * K);
    J.o_rxc[pi] = off;
    off += al((int64_t)J.rx[pi] * K);
    J.o_ryc[pi] = off;
    off += al((int64_t)J.ry[pi] * K);
    J.rx_off[pi] = J.tall_x[pi] ? J.o_gx[pi] : J.o_xf + P->afoff[pi];
    J.ldx[pi] = J.tall_x[pi] ? (int)K : (int)P->ldk[pi];
    J.ry_off[pi] = J.tall_y[pi] ? J.o_gy[pi] : J.o_yf + P->bfoff[pi];
    J.ldy[pi] = J.tall_y[pi] ? (int)K : (int)P->ldk[pi];
    J.trans[pi] = J.rx[pi] > J.ry[pi];  // rotate the shorter side
    J.nrot[pi] = J.trans[pi] ? J.ry[pi] : J.rx[pi];
    J.mlen[pi] = J.trans[pi] ? J.rx[pi] : J.ry[pi];
    J.o_m[pi] = off;
    off += al((int64_t)J.nrot[pi] * J.mlen[pi]);
    J.o_tf[pi] = off;
    off += al((int64_t)J.nrot[pi] * J.mlen[pi]);
    J.o_ms3[pi] = off;
    off += al((int64_t)J.nrot[pi] * J.mlen[pi]);
    // kept vectors and projectors (at most nrot of them)
    J.o_wk[pi] = off;
    off += al((int64_t)J.nrot[pi] * J.rx[pi]);
    J.o_zk[pi] = off;
    off += al((int64_t)J.nrot[pi] * J.ry[pi]);
    J.o_px[pi] = off;
    off += al((int64_t)J.nrot[pi] * K);
    J.o_qy[pi] = off;
    off += al((int64_t)J.nrot[pi] * K);
    J.o_sc[pi] = off;
    off += al(J.nrot[pi]);
  }
  J.ws_n = off;
  return FTN_OK;
}

// Householder TSQR jobs of the tall sides, by tree level: level 0 factors
// every chunk into its own slot; level l >= 1 merges slot c + 2^(l-1) into
// slot c for every c that is a multiple of 2^l (the merged factor is upper
// triangular, its zero prefix skipped).  levels[l] receives the jobs.
void cj_qr(CJob& J, std::vector<std::vector<QrJob>>& levels) {
  const TdPlan* P = J.P.get();
  auto side = [&](int K, int64_t rows, int64_t src, int64_t ld, int64_t slots, int64_t L, int nchunk) {
    if (nchunk == 0) return;
    if (levels.empty()) levels.resize(1);
    for (int c = 0; c < nchunk; ++c) {
      const int64_t r0 = (int64_t)c * L;
      levels[0].push_back({J.ws + src + r0 * ld, J.ws + slots + (int64_t)c * K * K, std::min(L, rows - r0), ld, K, 0,
                           0});
    }
    for (int l = 1; (1 << (l - 1)) < nchunk; ++l) {
      if ((int)levels.size() <= l) levels.resize(l + 1);
      const int h = 1 << (l - 1);
      for (int c = 0; c + h < nchunk; c += 2 * h)
        levels[l].push_back({J.ws + slots + (int64_t)(c + h) * K * K, J.ws + slots + (int64_t)c * K * K, K, K, K, 1,
                             1});
    }
  };
  for (int pi = 0; pi < 2; ++pi) {
    const int K = (int)P->K[pi];
    if (K == 0) continue;
    if (J.tall_x[pi] && P->M[pi] > 0)
      side(K, P->M[pi], J.o_xf + P->afoff[pi], P->ldk[pi], J.o_gx[pi], J.qr_lx[pi], J.qr_px[pi]);
    if (J.tall_y[pi] && P->N[pi] > 0)
      side(K, P->N[pi], J.o_yf + P->bfoff[pi], P->ldk[pi], J.o_gy[pi], J.qr_ly[pi], J.qr_py[pi]);
  }
}

// After the row counts: the compacted R factors and the core's shape.
ftn_status cj_counts(CJob& J, const int* hc) {
  const TdPlan* P = J.P.get();
  for (int pi = 0; pi < 2; ++pi) {
    const int K = (int)P->K[pi];
    if (K == 0 || J.rx[pi] == 0 || J.ry[pi] == 0) {
      J.rx[pi] = J.ry[pi] = 0;
      continue;
    }
    if (hc[2 * pi] < 0 || hc[2 * pi] > J.rx[pi] || hc[2 * pi + 1] < 0 || hc[2 * pi + 1] > J.ry[pi])
      return set_error(FTN_EINVAL, "internal error: R factor row count");
    J.rx[pi] = hc[2 * pi];
    J.ry[pi] = hc[2 * pi + 1];
    J.rx_off[pi] = J.o_rxc[pi];
    J.ldx[pi] = K;
    J.ry_off[pi] = J.o_ryc[pi];
    J.ldy[pi] = K;
    J.trans[pi] = J.rx[pi] > J.ry[pi];  // rotate the shorter side
    J.nrot[pi] = J.trans[pi] ? J.ry[pi] : J.rx[pi];
    J.mlen[pi] = J.trans[pi] ? J.rx[pi] : J.ry[pi];
  }
  return FTN_OK;
}

// Pooled truncation from the singular values of both sectors (values, then
// the sweep count, per sector at sv + s_off).
void cj_truncate(CJob& J, const double* sv) {
  std::vector<CJob::Cand> cand;
  double smax = 0, total = 0;
  int sweeps_used = 0;
  for (int pi = 0; pi < 2; ++pi) {
    if (!J.nrot[pi]) continue;
    const double* s = sv + J.s_off[pi];
    int sw = 0;
    std::memcpy(&sw, s + J.nrot[pi], sizeof(int));
    sweeps_used = std::max(sweeps_used, sw);
    for (int i = 0; i < J.nrot[pi]; ++i) {
      cand.push_back({s[i], pi, i});
      smax = std::max(smax, s[i]);
      total += s[i] * s[i];
    }
  }
  std::stable_sort(cand.begin(), cand.end(), [](const CJob::Cand& a, const CJob::Cand& b) {
    if (a.s != b.s) return a.s > b.s;
    if (a.pi != b.pi) return a.pi < b.pi;
    return a.idx < b.idx;
  });
  const double zero_tol = 1e-14 * smax;
  int rank_s[2] = {0, 0};
  for (auto& c : cand)
    if (c.s > zero_tol) rank_s[c.pi]++;
  double disc = 0;
  J.kept.clear();
  for (size_t i = 0; i < cand.size(); ++i) {
    if ((int)J.kept.size() < J.it->chi && cand[i].s > zero_tol)
      J.kept.push_back(cand[i]);
    else
      disc += cand[i].s * cand[i].s;
  }
  J.k[0] = J.k[1] = 0;
  for (auto& c : J.kept) J.k[c.pi]++;
  if (ftn_compress_info* info = J.it->info) {
    info->kept[0] = J.k[0];
    info->kept[1] = J.k[1];
    info->rank[0] = rank_s[0];
    info->rank[1] = rank_s[1];
    info->discarded_sq = disc;
    info->total_sq = total;
    info->s_max = smax;
    info->s_cut = J.kept.empty() ? 0.0 : J.kept.back().s;
    info->s_next = J.kept.size() < cand.size() ? cand[J.kept.size()].s : 0.0;
    info->jacobi_sweeps = sweeps_used;
  }
}

}  // namespace

// Batched compression: every stage of every job contributes to one launch
// per kernel; two host synchronisations per batch (the R-factor row counts
// and the singular values).
ftn_status compress_batch(ftn_ctx ctx, std::vector<CompressItem>& items) {
  if (!ctx) return set_error(FTN_EINVAL, "null argument");
  if (items.empty()) return FTN_OK;
  std::vector<CJob> jobs(items.size());
  int64_t total = 0;
  for (size_t i = 0; i < items.size(); ++i) {
    jobs[i].it = &items[i];
    FTN_TRY(cj_prepare(ctx, jobs[i]));
    jobs[i].ws_off = total;
    total += jobs[i].ws_n;
  }
  // shared small buffers after the jobs' workspaces: [row counts: 4 ints per job | singular values]
  int64_t s_total = 0;
  for (CJob& J : jobs)
    for (int pi = 0; pi < 2; ++pi) {
      J.s_off[pi] = s_total;
      s_total += J.nrot[pi] + 1;  // values, then the sweep count
    }
  const int64_t cnt_words = ((int64_t)jobs.size() * 4 * (int64_t)sizeof(int) + 7) / 8;
  double* ws = (double*)workspace(ctx, (size_t)(total + cnt_words + s_total + 32) * 8);
  if (!ws) return set_error(FTN_ENOMEM, "workspace allocation failed");
  for (CJob& J : jobs) J.ws = ws + J.ws_off;
  int* cnt = (int*)(ws + total);
  double* sbuf = ws + total + cnt_words;

  // ---- 1. fused matrices ----
  {
    PermBatch pb;
    for (CJob& J : jobs) {
      const TdPlan* P = J.P.get();
      pb.add(P->ja, P->ta, P->sa, J.it->X->data, J.ws + J.o_xf);
      pb.add(P->jb, P->tb, P->sb, J.it->Y->data, J.ws + J.o_yf);
    }
    FTN_TRY(flush_perm(ctx, pb, FTN_F64, PERM_SAME, 0));
  }
  // ---- 2. R factors by Householder TSQR (one launch per tree level) ----
  {
    std::vector<std::vector<QrJob>> levels;
    for (CJob& J : jobs) cj_qr(J, levels);
    int kmax = 0;
    for (auto& lv : levels)
      for (const QrJob& q : lv) kmax = std::max(kmax, q.K);
    const size_t smem = (size_t)QR_ROWS * kmax * sizeof(double);
    if (smem > 48 * 1024) FTN_CUDA(cudaFuncSetAttribute(qr_stream_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        (int)(QR_ROWS * LA_MAX_DIM * sizeof(double))));
    for (auto& lv : levels) {
      if (lv.empty()) continue;
      DevBuf t_qr(ctx);
      FTN_TRY(put_table(ctx, lv, &t_qr.p));
      const int rec = prof_begin(ctx, "householder_qr", 0, 0);
      qr_stream_kernel<<<(unsigned)lv.size(), QR_THREADS, smem, ctx->stream>>>((const QrJob*)t_qr.p);
      ctx->launches += 1;
      FTN_CUDA(cudaGetLastError());
      prof_end(ctx, rec);
    }
  }
  // ---- 2b. nonzero rows of the R factors (one synchronisation for the counts) ----
  {
    std::vector<CompactJob> cj;
    for (size_t q = 0; q < jobs.size(); ++q) {
      CJob& J = jobs[q];
      for (int pi = 0; pi < 2; ++pi) {
        const int K = (int)J.P->K[pi];
        if (K == 0 || J.rx[pi] == 0 || J.ry[pi] == 0) continue;
        cj.push_back({J.ws + J.rx_off[pi], J.ws + J.o_rxc[pi], cnt + 4 * q + 2 * pi, J.rx[pi], K, J.ldx[pi]});
        cj.push_back({J.ws + J.ry_off[pi], J.ws + J.o_ryc[pi], cnt + 4 * q + 2 * pi + 1, J.ry[pi], K, J.ldy[pi]});
      }
    }
    std::vector<int> hc(4 * jobs.size(), 0);
    if (!cj.empty()) {
      DevBuf t_cj(ctx);
      FTN_TRY(put_table(ctx, cj, &t_cj.p));
      FTN_CUDA(cudaMemsetAsync(cnt, 0, hc.size() * sizeof(int), ctx->stream));
      compact_rows_kernel<<<(unsigned)cj.size(), 256, 0, ctx->stream>>>((const CompactJob*)t_cj.p);
      ctx->launches += 1;
      FTN_CUDA(cudaGetLastError());
      FTN_CUDA(cudaMemcpyAsync(hc.data(), cnt, hc.size() * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
      FTN_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    for (size_t q = 0; q < jobs.size(); ++q) FTN_TRY(cj_counts(jobs[q], hc.data() + 4 * q));
  }
  // ---- 3. core M = R_X R_Y^T (stored with the rotated side as rows) and SVD ----
  {
    GemmF64Batch gb(ctx);
    std::vector<SvdJob> svd;
    for (CJob& J : jobs) {
      std::vector<GemmProb> mg;
      for (int pi = 0; pi < 2; ++pi) {
        const int K = (int)J.P->K[pi];
        if (K == 0 || J.rx[pi] == 0 || J.ry[pi] == 0) {
          J.nrot[pi] = 0;
          continue;
        }
        GemmProb g = make_prob(J.rx[pi], J.ry[pi], K, J.rx_off[pi], J.ldx[pi], 1, J.ry_off[pi], J.ldy[pi], 1);
        if (!J.trans[pi])
          gemm_plain_output(g, J.o_m[pi], J.ry[pi]);  // M: rx x ry
        else {
          gemm_plain_output(g, J.o_m[pi], 0);  // M^T: ry x rx  (element (i, j) at j * rx + i)
          g.rstr[0] = 1;
          g.cstr[0] = J.rx[pi];
        }
        mg.push_back(g);
        double* s = sbuf + J.s_off[pi];
        svd.push_back({J.ws + J.o_m[pi], J.ws + J.o_tf[pi], s, (int*)(s + J.nrot[pi]), J.nrot[pi], J.mlen[pi]});
      }
      FTN_TRY(add_gemm_set(gb, mg, J.ws, J.ws, J.ws, J.ws_n, J.ws_n, J.ws_n));
    }
    FTN_TRY(flush_gemm_f64(gb));
    if (!svd.empty()) {
      // rows up to 32 * SVDC_MAX_E long whose cluster share fits in shared
      // memory go to the cluster kernel (one launch; its arithmetic does not
      // depend on the cluster size or row length it is launched with, so a
      // decomposition does not depend on the other jobs of the batch), the
      // others to the single-CTA one
      const int cmax = svd_cluster_max(ctx);
      std::vector<SvdJob> small, big;
      int e_max = 1, c_use = 1;
      for (const SvdJob& j : svd) {
        const int np = j.n + (j.n & 1);
        int c = 1;
        while (c < cmax && c * SVDC_WARPS < np / 2) c *= 2;
        while (c < cmax && (int64_t)((j.n + c - 1) / c) * j.m * 8 > SVDC_SMEM_BYTES) c *= 2;
        if (j.m > 32 * SVDC_MAX_E || (int64_t)((j.n + c - 1) / c) * j.m * 8 > SVDC_SMEM_BYTES) {
          big.push_back(j);
          continue;
        }
        small.push_back(j);
        c_use = std::max(c_use, c);
        int e = 1;
        while (32 * e < j.m) e *= 2;
        e_max = std::max(e_max, e);
      }
      std::vector<SvdJob> all(small);
      all.insert(all.end(), big.begin(), big.end());
      DevBuf t_svd(ctx);
      FTN_TRY(put_table(ctx, all, &t_svd.p));
      const int rec = prof_begin(ctx, "svd_jacobi", 0, 0);
      if (!small.empty()) {
        size_t smem = 0;
        for (const SvdJob& j : small) smem = std::max(smem, (size_t)((j.n + c_use - 1) / c_use) * j.m * 8);
        FTN_TRY(launch_svd_cluster(ctx, (const SvdJob*)t_svd.p, (int)small.size(), c_use, e_max, smem));
      }
      if (!big.empty()) {
        svd_rows_global_kernel<<<(unsigned)big.size(), LA_THREADS, 0, ctx->stream>>>((const SvdJob*)t_svd.p +
                                                                                   small.size());
        ctx->launches += 1;
        FTN_CUDA(cudaGetLastError());
      }
      prof_end(ctx, rec);
    }
  }
  // ---- 4. pooled truncation (one synchronisation) ----
  {
    std::vector<double> sv(s_total + 1);
    if (s_total) FTN_CUDA(cudaMemcpyAsync(sv.data(), sbuf, s_total * 8, cudaMemcpyDeviceToHost, ctx->stream));
    FTN_CUDA(cudaStreamSynchronize(ctx->stream));
    for (CJob& J : jobs) cj_truncate(J, sv.data());
  }
  // ---- 5. projectors and the new tensors ----
  // m-side vectors (the orthogonalised rows' direction) come from T_f rows;
  // n-side vectors as T u_j / s_j by one GEMM with the untouched T.  Both are
  // wanted scaled by s^{-1/2}: MS = T_f row * s^{-3/2}, MS3 = T_f row * s^{-5/2}
  // and NS = MS3 T^T, whose rows are then re-orthogonalised (orth_rows_kernel).
  // Without transposition the m side is the right (ry) side of M, with it the
  // left (rx) side.
  {
    std::vector<GatherJob> gat;
    for (CJob& J : jobs) {
      int pos[2] = {0, 0};
      for (auto& c : J.kept) {
        const int pi = c.pi, j = pos[pi]++;
        const double* row = J.ws + J.o_tf[pi] + (int64_t)c.idx * J.mlen[pi];
        const double is = 1.0 / sqrt(c.s);
        GatherJob g;
        g.left = row;
        g.nl = J.mlen[pi];
        g.sl = is / c.s;
        g.right = row;
        g.nr = J.mlen[pi];
        g.sr = is / (c.s * c.s);
        g.dl = J.ws + (J.trans[pi] ? J.o_wk[pi] : J.o_zk[pi]) + (int64_t)j * J.mlen[pi];
        g.dr = J.ws + J.o_ms3[pi] + (int64_t)j * J.mlen[pi];
        g.dsc = J.ws + J.o_sc[pi] + j;
        g.sc = is;
        gat.push_back(g);
      }
    }
    if (!gat.empty()) {
      DevBuf t_gat(ctx);
      FTN_TRY(put_table(ctx, gat, &t_gat.p));
      gather_kernel<<<(unsigned)gat.size(), 128, 0, ctx->stream>>>((const GatherJob*)t_gat.p);
      ctx->launches += 1;
      FTN_CUDA(cudaGetLastError());
    }
  }
  {
    // NS[j, r] = sum_c MS3[j, c] T[r, c]   (k x nrot)
    GemmF64Batch gb(ctx);
    for (CJob& J : jobs) {
      std::vector<GemmProb> nside;
      for (int pi = 0; pi < 2; ++pi) {
        if (J.k[pi] == 0) continue;
        GemmProb g = make_prob(J.k[pi], J.nrot[pi], J.mlen[pi], J.o_ms3[pi], J.mlen[pi], 1, J.o_m[pi], J.mlen[pi], 1);
        gemm_plain_output(g, J.trans[pi] ? J.o_zk[pi] : J.o_wk[pi], J.nrot[pi]);
        nside.push_back(g);
      }
      FTN_TRY(add_gemm_set(gb, nside, J.ws, J.ws, J.ws, J.ws_n, J.ws_n, J.ws_n));
    }
    FTN_TRY(flush_gemm_f64(gb));
  }
  {
    // the n-side vectors re-orthogonalised against those of larger singular value
    std::vector<OrthJob> orth;
    for (CJob& J : jobs)
      for (int pi = 0; pi < 2; ++pi)
        if (J.k[pi] > 1)
          orth.push_back({J.ws + (J.trans[pi] ? J.o_zk[pi] : J.o_wk[pi]), J.ws + J.o_sc[pi], J.k[pi], J.nrot[pi]});
    if (!orth.empty()) {
      DevBuf t_orth(ctx);
      FTN_TRY(put_table(ctx, orth, &t_orth.p));
      orth_rows_kernel<<<(unsigned)orth.size(), 256, 0, ctx->stream>>>((const OrthJob*)t_orth.p);
      ctx->launches += 1;
      FTN_CUDA(cudaGetLastError());
    }
  }
  {
    // P_X^T = Z_k R_Y (k x K) and Q_Y^T = W_k R_X (k x K)
    GemmF64Batch gb(ctx);
    for (CJob& J : jobs) {
      std::vector<GemmProb> proj;
      for (int pi = 0; pi < 2; ++pi) {
        const int K = (int)J.P->K[pi];
        if (J.k[pi] == 0) continue;
        GemmProb a = make_prob(J.k[pi], K, J.ry[pi], J.o_zk[pi], J.ry[pi], 1, J.ry_off[pi], 1, J.ldy[pi]);
        gemm_plain_output(a, J.o_px[pi], K);
        proj.push_back(a);
        GemmProb b = make_prob(J.k[pi], K, J.rx[pi], J.o_wk[pi], J.rx[pi], 1, J.rx_off[pi], 1, J.ldx[pi]);
        gemm_plain_output(b, J.o_qy[pi], K);
        proj.push_back(b);
      }
      FTN_TRY(add_gemm_set(gb, proj, J.ws, J.ws, J.ws, J.ws_n, J.ws_n, J.ws_n));
    }
    FTN_TRY(flush_gemm_f64(gb));
  }
  // new tensors: X' = [free_X | new(-)], Y' = [new(+) | free_Y].  Every
  // element of every block is written by one GEMM below: a block has nonzero
  // size only if its sector of the new leg kept states (k > 0), and then its
  // free-row (free-column) sector is one problem of the set.
  struct Outs {
    std::vector<CJob>& v;
    bool ok = false;
    ~Outs() {
      if (ok) return;
      for (CJob& J : v) {
        ftn_tensor_free(J.Xn);
        ftn_tensor_free(J.Yn);
        J.Xn = J.Yn = nullptr;
      }
    }
  } outs{jobs};
  {
    GemmF64Batch gb(ctx);
    for (CJob& J : jobs) {
      const TdPlan* P = J.P.get();
      ftn_tensor X = J.it->X, Y = J.it->Y;
      int32_t xd0[MAXR], xd1[MAXR], yd0[MAXR], yd1[MAXR];
      uint8_t xdu[MAXR], ydu[MAXR];
      for (int j = 0; j < P->nfa; ++j)
        xd0[j] = X->d0[P->fa[j]], xd1[j] = X->d1[P->fa[j]], xdu[j] = X->dual[P->fa[j]];
      xd0[P->nfa] = J.k[0], xd1[P->nfa] = J.k[1], xdu[P->nfa] = 1;
      yd0[0] = J.k[0], yd1[0] = J.k[1], ydu[0] = 0;
      for (int j = 0; j < P->nfb; ++j)
        yd0[j + 1] = Y->d0[P->fb[j]], yd1[j + 1] = Y->d1[P->fb[j]], ydu[j + 1] = Y->dual[P->fb[j]];
      FTN_TRY(make_tensor(ctx, P->nfa + 1, xd0, xd1, xdu, X->parity, FTN_F64, &J.Xn));
      FTN_TRY(make_tensor(ctx, P->nfb + 1, yd0, yd1, ydu, Y->parity, FTN_F64, &J.Yn));
      std::vector<GemmProb> fx, fy;
      for (int pi = 0; pi < 2; ++pi) {
        if (J.k[pi] == 0) continue;
        const int K = (int)P->K[pi];
        const int rho = X->parity ^ pi, sig = Y->parity ^ pi;
        for (uint32_t mA = 0; mA < (1u << P->nfa); ++mA) {
          if ((popc(mA) & 1) != rho || P->rowsz[pi][mA] == 0) continue;
          const uint32_t mask = mA | ((uint32_t)pi << P->nfa);
          GemmProb g = make_prob((int)P->rowsz[pi][mA], J.k[pi], K,
                                 J.o_xf + P->afoff[pi] + P->rowoff[pi][mA] * P->ldk[pi], P->ldk[pi], 1, J.o_px[pi], K,
                                 1);
          gemm_plain_output(g, J.Xn->offsets[mask >> 1], J.k[pi]);
          fx.push_back(g);
        }
        for (uint32_t mB = 0; mB < (1u << P->nfb); ++mB) {
          if ((popc(mB) & 1) != sig || P->colsz[pi][mB] == 0) continue;
          const uint32_t mask = (uint32_t)pi | (mB << 1);
          const int Cm = (int)P->colsz[pi][mB];
          GemmProb g = make_prob(Cm, J.k[pi], K, J.o_yf + P->bfoff[pi] + P->coloff[pi][mB] * P->ldk[pi], P->ldk[pi],
                                 1, J.o_qy[pi], K, 1);
          gemm_plain_output(g, J.Yn->offsets[mask >> 1], 0);  // written transposed: (new, free)
          g.rstr[0] = 1;
          g.cstr[0] = Cm;
          fy.push_back(g);
        }
      }
      FTN_TRY(add_gemm_set(gb, fx, J.ws, J.ws, (double*)J.Xn->data, J.ws_n, J.ws_n, J.Xn->numel));
      FTN_TRY(add_gemm_set(gb, fy, J.ws, J.ws, (double*)J.Yn->data, J.ws_n, J.ws_n, J.Yn->numel));
    }
    FTN_TRY(flush_gemm_f64(gb));
  }
  outs.ok = true;
  for (CJob& J : jobs) {
    ftn_tensor_free(J.it->X);
    ftn_tensor_free(J.it->Y);
    J.it->X = J.Xn;
    J.it->Y = J.Yn;
  }
  return FTN_OK;
}

ftn_status compress_impl(ftn_ctx ctx, ftn_tensor* pX, ftn_tensor* pY, int n, const int* ax, const int* ay, int chi,
                         int arrows, ftn_compress_info* info) {
  if (!ctx || !pX || !pY || !*pX || !*pY || (n > 0 && (!ax || !ay))) return set_error(FTN_EINVAL, "null argument");
  if (n < 1) return set_error(FTN_EINVAL, "a bond needs at least one leg pair");
  if (n > MAXR) return set_error(FTN_EINVAL, "too many bond legs");
  std::vector<CompressItem> items(1);
  CompressItem& it = items[0];
  it.X = *pX;
  it.Y = *pY;
  it.n = n;
  for (int i = 0; i < n; ++i) it.ax[i] = ax[i], it.ay[i] = ay[i];
  it.chi = chi;
  it.arrows = arrows;
  it.info = info;
  FTN_TRY(compress_batch(ctx, items));
  *pX = it.X;
  *pY = it.Y;
  return FTN_OK;
}

}  // namespace ftn

using namespace ftn;

extern "C" ftn_status ftn_compress(ftn_ctx ctx, ftn_tensor* X, ftn_tensor* Y, int n, const int* axes_x,
                                   const int* axes_y, int chi, int arrows, ftn_compress_info* info) {
  return compress_impl(ctx, X, Y, n, axes_x, axes_y, chi, arrows, info);
}
