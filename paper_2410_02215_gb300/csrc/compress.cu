// Bond compression ftn_compress (Sec. II.A: symmetric QR/SVD with the chi
// largest singular values pooled over all symmetry blocks; Sec. II.B: the
// decomposition runs after transposing into row | column order).
//
// GPU pipeline, FP64 throughout, per bond-parity sector pi:
//   1. sign-permute X -> X_pi = [free_X | bond] and Y -> Y_pi^T = [free_Y | bond]
//      (the fused layouts of the tensordot, bond parity of the arrow folded in);
//   2. R factors with R^T R = X_pi^T X_pi (resp. Y_pi Y_pi^T): Gram matrix by
//      the FP64 GEMM and a semi-definite Cholesky.  A Gram matrix resolves
//      singular values only down to ~1e-8 of the largest, so a side whose
//      Cholesky meets a pivot that is neither exactly zero nor at least 1e-6
//      of the largest diagonal is factored again by Householder QR (only R is
//      formed: each CTA streams a chunk of rows through shared memory into
//      its own triangular factor, and a binary tree of the same kernel merges
//      the chunks' factors, TSQR), which is backward stable whatever the
//      condition; a side with no more rows than bond states uses the matrix
//      itself (X_pi = I * X_pi);
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

struct CholJob {
  double* G;  // n x n row-major, symmetric; replaced by R (upper, R^T R = G)
  int n;
  int* flag;      // bit 0: a pivot in (1e-12, 1e-6) of the largest diagonal; bit 1: a nonzero pivot dropped
  double* trace;  // receives trace(G) = |underlying matrix|_F^2
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

__device__ __forceinline__ double block_max(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[32] = v;
  }
  __syncthreads();
  return red[32];
}

// Semi-definite Cholesky G = L L^T (right-looking); a pivot at or below
// 1e-12 * max(diag G) marks a numerically dependent direction (a singular
// value of the underlying matrix below 1e-6 of its largest, where a Gram
// matrix carries only rounding noise) whose row of R is set to zero.
// Writes R = L^T (upper triangle, zeros below).  The Gram matrix resolves a
// direction of the underlying matrix only down to ~1e-8 of its largest
// singular value.  The factor is therefore kept as it is when every pivot is
// exactly zero (an empty column) or at least 1e-6 of the largest diagonal.
// A pivot between 1e-12 and 1e-6 (bit 0 of *flag) sends the side to the
// Householder QR; dropped pivots that are not exactly zero (bit 1) mean
// columns dependent on the kept ones up to rounding -- or directions the Gram
// matrix cannot see -- and are settled by the residual test of
// dropped_residual_kernel.
__global__ void __launch_bounds__(LA_THREADS) chol_kernel(const CholJob* jobs) {
  __shared__ double red[33];
  __shared__ double piv;
  const CholJob jb = jobs[blockIdx.x];
  double* G = jb.G;
  const int n = jb.n;
  double dmax = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) dmax = fmax(dmax, G[(int64_t)i * n + i]);
  dmax = block_max(dmax, red);
  const double tol = 1e-12 * dmax;
  if (threadIdx.x == 0 && jb.trace) {
    double tr = 0.0;
    for (int i = 0; i < n; ++i) tr += G[(int64_t)i * n + i];
    *jb.trace = tr;
  }
  int fl = 0;
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      const double d = G[(int64_t)j * n + j];
      piv = d > tol ? sqrt(d) : 0.0;
      G[(int64_t)j * n + j] = piv;
      if (d > tol && d < 1e-6 * dmax) fl |= 1;
      if (!(d > tol) && d != 0.0) fl |= 2;
    }
    __syncthreads();
    const double p = piv;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x)
      G[(int64_t)i * n + j] = p > 0.0 ? G[(int64_t)i * n + j] / p : 0.0;
    __syncthreads();
    const int rest = n - j - 1;
    const int64_t cnt = (int64_t)rest * rest;
    for (int64_t e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int i = j + 1 + (int)(e / rest), k = j + 1 + (int)(e % rest);
      if (k <= i) G[(int64_t)i * n + k] -= G[(int64_t)i * n + j] * G[(int64_t)k * n + j];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && fl && jb.flag) *jb.flag = fl;
  // R = L^T in place
  const int64_t tot = (int64_t)n * n;
  for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
    const int i = (int)(e / n), k = (int)(e % n);
    if (i < k) {
      G[(int64_t)i * n + k] = G[(int64_t)k * n + i];
      G[(int64_t)k * n + i] = 0.0;
    }
  }
}

constexpr int QR_ROWS = 16;      // rows of src per pass when K > QR_WIDE_K
constexpr int QR_ROWS_WIDE = 32; // rows per pass otherwise (one per lane of warp 0 in the norm)
constexpr int QR_WIDE_K = 512;   // largest K streamed 32 rows at a time (32 x 512 doubles = 128 KB)
constexpr int QR_RSMEM_K = 128;  // largest K whose factor stays in shared memory (128 KB)
constexpr int QR_THREADS = 128;

// Householder QR, R factor only (Sec. II.A: the QR of each symmetry block).
// Rows arrive in blocks of ROWS held in shared memory.  For column j with
// x = [a; b] = [R_jj; B(:, j)] the reflector H = I - tau v v^T, v = [1; b / (a
// - beta)], beta = -sign(a) |x|, tau = (beta - a) / beta in [1, 2], maps x to
// [beta; 0] and is applied to the trailing columns of R row j and of the
// block (the form of LAPACK's dlarfg; |x| is taken after scaling by max|x|
// whenever a square or product could leave the normal range, so no
// intermediate overflows or underflows, however small b has become).  Row j of R is read
// and written only at step j: R stays in shared memory when RSMEM (K <=
// QR_RSMEM_K), else in global memory (L2-resident; each access is one
// coalesced row).  A column whose block part is zero, or below 2^-960 in
// magnitude, needs no reflector (this also skips the zero prefix of
// triangular sources).  Once a short block's rank is absorbed its rows hold
// only rounding noise, which every further group of reflectors shrinks by
// ~2^-52: that is where such tiny columns arise.
template <int ROWS, bool RSMEM>
__global__ void __launch_bounds__(QR_THREADS) qr_stream_kernel(const QrJob* jobs) {
  extern __shared__ double qsm[];  // [R (K x K) when RSMEM] then the block (ROWS x K, row-major)
  __shared__ double refl[2];       // tau, 1 / (a - beta)
  __shared__ int skip;
  const QrJob J = jobs[blockIdx.x];
  const int K = J.K, t = threadIdx.x, lane = t & 31, warp = t >> 5;
  double* R = RSMEM ? qsm : J.R;
  double* qb = RSMEM ? qsm + (size_t)K * K : qsm;
  const int64_t kk = (int64_t)K * K;
  if (!J.init)
    for (int64_t e = t; e < kk; e += blockDim.x) R[e] = 0.0;
  else if (RSMEM)
    for (int64_t e = t; e < kk; e += blockDim.x) R[e] = J.R[e];
  for (int64_t r0 = 0; r0 < J.rows; r0 += ROWS) {
    const int nb = (int)(J.rows - r0 < ROWS ? J.rows - r0 : ROWS);
    __syncthreads();  // the previous block's last column is done (and R is set up)
    for (int e = t; e < ROWS * K; e += blockDim.x) {
      const int i = e / K, c = e - i * K;
      qb[e] = i < nb ? J.src[(r0 + i) * J.ld + c] : 0.0;
    }
    __syncthreads();
    const int j0 = J.tri ? (int)(r0 < K ? r0 : K) : 0;
    for (int j = j0; j < K; ++j) {
      if (warp == 0) {
        const double bj = lane < ROWS ? qb[lane * K + j] : 0.0;
        double ss = bj * bj;
        for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (lane == 0) {
          const double a = R[(int64_t)j * K + j];
          int sk = 0;
          if (ss >= 0x1p-900 && ss <= 0x1p900 && fabs(a) <= 0x1p450) {
            // every square and product below stays in the normal range
            const double nrm = sqrt(fma(a, a, ss));
            const double beta = a > 0.0 ? -nrm : nrm;
            const double d = a - beta;  // |d| >= nrm, no cancellation
            const double r = 1.0 / (beta * d);
            refl[0] = -(d * d) * r;  // (beta - a) / beta
            refl[1] = beta * r;      // 1 / (a - beta)
            R[(int64_t)j * K + j] = beta;
          } else {
            // rescaled by the largest magnitude of the column
            double mx = 0.0;
            for (int i = 0; i < ROWS; ++i) mx = fmax(mx, fabs(qb[i * K + j]));
            if (mx > 0x1p-960) {
              const double sc = fmax(mx, fabs(a)), rs = 1.0 / sc, as = a * rs;
              double s2 = 0.0;
              for (int i = 0; i < ROWS; ++i) {
                const double u = qb[i * K + j] * rs;
                s2 = fma(u, u, s2);
              }
              const double nrm = sc * sqrt(fma(as, as, s2));
              const double beta = a > 0.0 ? -nrm : nrm;
              const double d = a - beta;
              refl[0] = -d / beta;
              refl[1] = 1.0 / d;
              R[(int64_t)j * K + j] = beta;
            } else {
              sk = 1;
            }
          }
          skip = sk;
        }
      }
      __syncthreads();
      if (!skip) {
        const double tau = refl[0], id = refl[1];
        for (int c = j + 1 + t; c < K; c += blockDim.x) {
          double* rp = R + (int64_t)j * K + c;
          const double rjc = *rp;
          double w0 = 0.0, w1 = 0.0;
#pragma unroll
          for (int i = 0; i < ROWS; i += 2) {
            w0 = fma(qb[i * K + j], qb[i * K + c], w0);
            w1 = fma(qb[(i + 1) * K + j], qb[(i + 1) * K + c], w1);
          }
          const double w = tau * fma(w0 + w1, id, rjc);
          *rp = rjc - w;
          const double wv = w * id;
#pragma unroll
          for (int i = 0; i < ROWS; ++i) qb[i * K + c] = fma(-wv, qb[i * K + j], qb[i * K + c]);
        }
      }
      __syncthreads();
    }
  }
  if (RSMEM) {
    __syncthreads();
    for (int64_t e = t; e < kk; e += blockDim.x) J.R[e] = R[e];
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

// Residual test of a Gram factor with dropped pivots.  With S the kept
// pivots (R_jj > 0) and D the dropped ones, column d of T (K x K, row-major)
// is e_d - Z R[S, d] for d in D, where Z holds R_SS^{-1} on the rows S, and 0
// for d in S; then E = A T has the columns A_D - A_S R_SS^{-1} R_SD: what is
// left of each dropped column after removing its part in the span of the kept
// ones (R_SS^{-1} R_SD are the coefficients the Cholesky found for it).  E is
// formed from A by a GEMM, so |E| is accurate to rounding of A itself (the
// Gram matrix could only tell it down to ~1e-8 |A|).  Each warp takes a
// column; lanes hold the right-hand side and the back substitution runs over
// the kept indices below d.
struct ResidTJob {
  const double* R;  // K x K upper-triangular factor, zero rows for dropped pivots
  double* T;
  int K;
  int c0;  // first column of this job's 32
};

constexpr int RESID_SMEM_K = 128;  // largest K staged in shared memory (R^T: 128 KB)

template <bool SM>
__global__ void __launch_bounds__(128) dropped_residual_kernel(const ResidTJob* jobs) {
  extern __shared__ double rsm[];  // SM: R^T (K x K), 1 / R_ss (K), then one right-hand side (K) per warp
  const ResidTJob J = jobs[blockIdx.x];
  const int K = J.K, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* Rt = rsm;
  double* inv = rsm + (SM ? (size_t)K * K : 0);
  double* bw = inv + (SM ? K : 0) + (size_t)warp * K;
  if (SM) {
    for (int64_t e = threadIdx.x; e < (int64_t)K * K; e += blockDim.x) {
      const int i = (int)(e / K), c = (int)(e - (int64_t)i * K);
      Rt[(int64_t)c * K + i] = J.R[e];
    }
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
      const double r = J.R[(int64_t)i * K + i];
      inv[i] = r != 0.0 ? 1.0 / r : 0.0;
    }
    __syncthreads();
  }
  // R[i, s] and the solve's right-hand side, from shared memory or from the
  // output column itself
  auto Ris = [&](int i, int sc) { return SM ? Rt[(int64_t)sc * K + i] : J.R[(int64_t)i * K + sc]; };
  for (int d = J.c0 + warp; d < J.c0 + 32 && d < K; d += 4) {
    double* Tc = J.T + d;  // column d, stride K
    if (J.R[(int64_t)d * K + d] != 0.0) {
      for (int i = lane; i < K; i += 32) Tc[(int64_t)i * K] = 0.0;
      continue;
    }
    double* b = SM ? bw : nullptr;
    // b = R[0..d-1, d]; x_s = (b_s - sum_{s < s' < d} R[s, s'] x_s') / R_ss over kept s; T[s, d] = -x_s
    for (int i = lane; i < K; i += 32) {
      const double v = i < d ? Ris(i, d) : 0.0;
      if (SM) b[i] = v;
      else Tc[(int64_t)i * K] = v;
    }
    __syncwarp();
    for (int sc = d - 1; sc >= 0; --sc) {
      const double rss = SM ? 1.0 : J.R[(int64_t)sc * K + sc];
      const double bs = SM ? b[sc] : Tc[(int64_t)sc * K];
      const double xs = SM ? bs * inv[sc] : (rss != 0.0 ? bs / rss : 0.0);
      __syncwarp();
      if (SM) {
        if (lane == 0) b[sc] = -xs;
        if (xs != 0.0)
          for (int i = lane; i < sc; i += 32) b[i] = fma(-Ris(i, sc), xs, b[i]);
      } else {
        if (lane == 0) Tc[(int64_t)sc * K] = -xs;
        if (xs != 0.0)
          for (int i = lane; i < sc; i += 32) Tc[(int64_t)i * K] -= Ris(i, sc) * xs;
      }
      __syncwarp();
    }
    if (SM)
      for (int i = lane; i < K; i += 32) Tc[(int64_t)i * K] = i == d ? 1.0 : (i < d ? b[i] : 0.0);
    else if (lane == 0)
      Tc[(int64_t)d * K] = 1.0;
    __syncwarp();
  }
}

// Sum of squares of each job's n elements (one CTA per job, fixed order).
struct SumSqJob {
  const double* x;
  int64_t n;
  double* out;
};

__global__ void __launch_bounds__(256) sumsq_kernel(const SumSqJob* jobs) {
  __shared__ double red[8];
  const SumSqJob J = jobs[blockIdx.x];
  double q = 0.0;
  for (int64_t e = threadIdx.x; e < J.n; e += blockDim.x) q = fma(J.x[e], J.x[e], q);
  for (int o = 16; o; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = q;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    *J.out = t;
  }
}

struct CompactJob {
  const double* src;  // rows x cols, leading dimension ld
  double* dst;        // the nonzero rows, packed (leading dimension cols)
  int* count;         // number of nonzero rows
  int rows, cols, ld;
};

// Packs the rows of an R factor that are not identically zero (rows of
// dropped Cholesky pivots, or zero rows of a side used as its own
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

// Opt the Householder QR and residual-test kernels into their shared-memory
// sizes (once per process).
ftn_status setup_qr_kernels() {
  static std::once_flag once;
  static cudaError_t err = cudaSuccess;
  std::call_once(once, [] {
    const int big = (QR_RSMEM_K * QR_RSMEM_K + QR_ROWS_WIDE * QR_RSMEM_K) * 8;
    err = cudaFuncSetAttribute(qr_stream_kernel<QR_ROWS_WIDE, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(qr_stream_kernel<QR_ROWS_WIDE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 QR_ROWS_WIDE * QR_WIDE_K * 8);
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(qr_stream_kernel<QR_ROWS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 QR_ROWS * LA_MAX_DIM * 8);
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(dropped_residual_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (RESID_SMEM_K * RESID_SMEM_K + 5 * RESID_SMEM_K) * 8);
  });
  if (err != cudaSuccess) return cuda_error(err, "cudaFuncSetAttribute (Householder QR)");
  return FTN_OK;
}

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

// ---- adjoint (gradient) of the compression: small dense kernels ----------------
// The backward pass of ftn_compress_grad works per bond-parity sector on the
// forward's factors: R_X, R_Y (compacted), the Jacobi rows T_f = s_j x (unit
// vector), the kept vectors W = S^-1/2 U_k^T and Z = S^-1/2 V_k^T.  Products
// go through the FP64 GEMM; these kernels do the rest (one CTA per matrix).

// out[j, c] = in[j, c] / s[j] for s[j] > tol, 0 otherwise (rows x cols,
// contiguous rows): a singular direction at or below tol is left out of the
// rebuilt factors and falls into the complements the adjoint projects onto
struct RowDivJob {
  const double* in;
  double* out;
  const double* s;
  int rows, cols;
  double tol;
};
__global__ void __launch_bounds__(256) row_div_kernel(const RowDivJob* jobs) {
  const RowDivJob J = jobs[blockIdx.x];
  const int64_t n = (int64_t)J.rows * J.cols;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    const int j = (int)(e / J.cols);
    J.out[e] = J.s[j] > J.tol ? J.in[e] / J.s[j] : 0.0;
  }
}

// Cotangents of the thin SVD's factors from those of Z and W: for kept state
// j (Jacobi row i = idx[j]) du_i = s_i^-1/2 dW[j], dv_i = s_i^-1/2 dZ[j] and
// ds_i = -1/2 s_i^-3/2 (dZ[j] . v_i + dW[j] . u_i); zero for the others.
struct CotJob {
  const double* dZ;  // k x ry
  const double* dW;  // k x rx
  const double* Ut;  // r x rx (rows u_i)
  const double* Vt;  // r x ry
  const double* s;   // r (Jacobi order)
  const int* idx;    // k: Jacobi row of kept state j
  double* dUt;       // r x rx
  double* dVt;       // r x ry
  double* ds;        // r
  int k, r, rx, ry;
};
__global__ void __launch_bounds__(256) svd_cot_kernel(const CotJob* jobs) {
  const CotJob J = jobs[blockIdx.x];
  for (int64_t e = threadIdx.x; e < (int64_t)J.r * J.rx; e += blockDim.x) J.dUt[e] = 0.0;
  for (int64_t e = threadIdx.x; e < (int64_t)J.r * J.ry; e += blockDim.x) J.dVt[e] = 0.0;
  for (int e = threadIdx.x; e < J.r; e += blockDim.x) J.ds[e] = 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j < J.k; j += nw) {
    const int i = J.idx[j];
    const double si = J.s[i], a = 1.0 / sqrt(si);
    double dot = 0.0;
    for (int c = lane; c < J.rx; c += 32) {
      const double w = J.dW[(int64_t)j * J.rx + c];
      J.dUt[(int64_t)i * J.rx + c] = a * w;
      dot = fma(w, J.Ut[(int64_t)i * J.rx + c], dot);
    }
    for (int c = lane; c < J.ry; c += 32) {
      const double z = J.dZ[(int64_t)j * J.ry + c];
      J.dVt[(int64_t)i * J.ry + c] = a * z;
      dot = fma(z, J.Vt[(int64_t)i * J.ry + c], dot);
    }
    for (int o = 16; o; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
    if (lane == 0) J.ds[i] = -0.5 * dot * a / si;
  }
}

// The core of the thin-SVD adjoint (r x r, Jacobi order):
//   inner = (F o (X - X^T)) S + diag(ds) + S (F o (Y - Y^T)),
// X = U^T dU, Y = V^T dV, F_ij = 1 / (s_j^2 - s_i^2) for i != j with i or j
// kept (pairs of discarded states carry no cotangent) and neither left out
// (a direction left out belongs to the complements: its terms are those of
// the projections), 0 otherwise.
struct InnerJob {
  const double* X;
  const double* Y;
  const double* s;
  const double* ds;
  const int* kept;  // r flags: 1 kept, 0 discarded, -1 left out (singular value at rounding level)
  double* inner;
  int r;
};
__global__ void __launch_bounds__(256) svd_inner_kernel(const InnerJob* jobs) {
  const InnerJob J = jobs[blockIdx.x];
  const int r = J.r;
  for (int64_t e = threadIdx.x; e < (int64_t)r * r; e += blockDim.x) {
    const int i = (int)(e / r), j = (int)(e - (int64_t)i * r);
    double v = 0.0;
    if (i == j) {
      v = J.ds[i];
    } else if ((J.kept[i] > 0 || J.kept[j] > 0) && J.kept[i] >= 0 && J.kept[j] >= 0) {
      const double si = J.s[i], sj = J.s[j];
      const double f = 1.0 / ((sj - si) * (sj + si));
      const double xa = J.X[(int64_t)i * r + j] - J.X[(int64_t)j * r + i];
      const double ya = J.Y[(int64_t)i * r + j] - J.Y[(int64_t)j * r + i];
      v = f * (xa * sj + si * ya);
    }
    J.inner[e] = v;
  }
}

// out = a + sa * b (elementwise over n), or, with s set, out[j, c] = a[j, c]
// + sa * b[j, c] * sinv_j with sinv_j = 1 / s_j for kept rows, 0 otherwise.
struct AxpyJob {
  const double* a;
  const double* b;
  double* out;
  const double* s;
  const int* kept;
  int64_t n;
  int cols;
  double sa;
};
__global__ void __launch_bounds__(256) axpy_kernel(const AxpyJob* jobs) {
  const AxpyJob J = jobs[blockIdx.x];
  for (int64_t e = threadIdx.x; e < J.n; e += blockDim.x) {
    double f = J.sa;
    if (J.s) {
      const int j = (int)(e / J.cols);
      f = J.kept[j] > 0 ? f / J.s[j] : 0.0;
    }
    J.out[e] = (J.a ? J.a[e] : 0.0) + f * J.b[e];
  }
}

// C := copyltu(C) = tril(C) + tril(C, -1)^T (n x n, in place)
struct SqJob {
  double* C;
  const double* R;
  int n;
};
__global__ void __launch_bounds__(256) copyltu_kernel(const SqJob* jobs) {
  const SqJob J = jobs[blockIdx.x];
  for (int64_t e = threadIdx.x; e < (int64_t)J.n * J.n; e += blockDim.x) {
    const int i = (int)(e / J.n), j = (int)(e - (int64_t)i * J.n);
    if (i < j) J.C[e] = J.C[(int64_t)j * J.n + i];
  }
}

// C := R^-1 for an upper-triangular n x n R with nonzero diagonal: column j
// of the inverse by back substitution (one thread per column).
__global__ void __launch_bounds__(256) tri_inverse_kernel(const SqJob* jobs) {
  const SqJob J = jobs[blockIdx.x];
  const int n = J.n;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    for (int i = n - 1; i >= 0; --i) {
      double v = 0.0;
      if (i <= j) {
        v = i == j ? 1.0 : 0.0;
        for (int c = i + 1; c <= j; ++c) v = fma(-J.R[(int64_t)i * n + c], J.C[(int64_t)c * n + j], v);
        v /= J.R[(int64_t)i * n + i];
      }
      J.C[(int64_t)i * n + j] = v;
    }
  }
}

// Adjoint of a sign-permute job table: the forward wrote dst[dst position] =
// sign * src[src position] for every element of every job; this writes
// src[src position] = sign * dst[dst position] (one CTA per job).
__global__ void __launch_bounds__(256) perm_adjoint_kernel(const PermJob* jobs, const double* __restrict__ dst,
                                                           double* __restrict__ src) {
  const PermJob& J = jobs[blockIdx.x];
  const int nl = J.nI + J.nO + J.nB;
  int64_t total = 1;
  for (int l = 0; l < nl; ++l) total *= J.dim[l];
  const double sg = (double)J.sign;
  for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
    int64_t x = e, so = J.src_off, dof = J.dst_off;
    for (int l = nl - 1; l >= 0; --l) {
      const int64_t q = x / J.dim[l];
      const int64_t i = x - q * J.dim[l];
      so += i * J.sstr[l];
      dof += i * J.dstr[l];
      x = q;
    }
    src[so] = sg * dst[dof];
  }
}

// Rebuilt singular vectors (rows of v, length n) taken in the order ord[0],
// ord[1], ... (decreasing singular value): each orthogonalised twice against
// the ones before it by classical Gram-Schmidt and scaled to unit norm.  The
// n-side vectors core x v_j / s_j carry ~eps s_max / s_j of the directions of
// larger singular values, which the F-matrix terms of the adjoint would pick
// up; this removes them, as the forward does for its kept vectors.
// Rows moved between the core's row order and the order of decreasing
// singular values: dst row q = src row idx[q] (gather) or dst row idx[q] =
// src row q (scatter); rows of len doubles.
struct RowsJob {
  const double* src;
  double* dst;
  const int* idx;
  int nrows, len, scatter;
};
__global__ void __launch_bounds__(256) rows_move_kernel(const RowsJob* jobs) {
  const RowsJob J = jobs[blockIdx.x];
  for (int64_t e = threadIdx.x; e < (int64_t)J.nrows * J.len; e += blockDim.x) {
    const int q = (int)(e / J.len), c = (int)(e - (int64_t)q * J.len);
    const int64_t a = (int64_t)q * J.len + c, b = (int64_t)J.idx[q] * J.len + c;
    J.dst[J.scatter ? b : a] = J.src[J.scatter ? a : b];
  }
}

// G (n x n, row-major, symmetric positive definite, n <= ORTH_B) := L^{-1},
// G = L L^T with L lower triangular (Cholesky, column by column), the
// inverse by forward substitution, one column per thread.  A pivot that is
// not positive zeroes its row of the inverse.
constexpr int ORTH_B = 48;
struct CholInvJob {
  double* g;
  int n;
};
__global__ void __launch_bounds__(256) chol_inv_small_kernel(const CholInvJob* jobs) {
  __shared__ double L[ORTH_B][ORTH_B + 1];
  __shared__ double Y[ORTH_B][ORTH_B + 1];
  const CholInvJob J = jobs[blockIdx.x];
  const int n = J.n, t = threadIdx.x;
  for (int e = t; e < n * n; e += blockDim.x) L[e / n][e % n] = J.g[e];
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (t == 0) L[j][j] = L[j][j] > 0.0 ? sqrt(L[j][j]) : 0.0;
    __syncthreads();
    const double dj = L[j][j];
    for (int i = j + 1 + t; i < n; i += blockDim.x) L[i][j] = dj > 0.0 ? L[i][j] / dj : 0.0;
    __syncthreads();
    const int w = n - j - 1;
    for (int e = t; e < w * w; e += blockDim.x) {
      const int a = j + 1 + e / w, b = j + 1 + e % w;
      if (b <= a) L[a][b] = fma(-L[a][j], L[b][j], L[a][b]);
    }
    __syncthreads();
  }
  for (int c = t; c < n; c += blockDim.x) {
    for (int i = 0; i < n; ++i) {
      if (i < c || L[i][i] == 0.0) {
        Y[i][c] = 0.0;
        continue;
      }
      double v = i == c ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) v = fma(-L[i][k], Y[k][c], v);
      Y[i][c] = v / L[i][i];
    }
  }
  __syncthreads();
  for (int e = t; e < n * n; e += blockDim.x) J.g[e] = Y[e / n][e % n];
}

// out[m, c] += a[m, c] (rows x cols; row strides lda, ldo)
struct Add2Job {
  const double* a;
  double* out;
  int rows, cols;
  int64_t lda, ldo;
};
// (grid: jobs x row slices; slice y takes rows y, y + gridDim.y, ...)
__global__ void __launch_bounds__(256) add2_kernel(const Add2Job* jobs) {
  const Add2Job J = jobs[blockIdx.x];
  for (int m = blockIdx.y; m < J.rows; m += gridDim.y)
    for (int c = threadIdx.x; c < J.cols; c += blockDim.x) J.out[m * J.ldo + c] += J.a[m * J.lda + c];
}

template <typename T>
ftn_status launch_jobs(ftn_ctx ctx, void (*k)(const T*), const std::vector<T>& jobs, unsigned slices = 1) {
  if (jobs.empty()) return FTN_OK;
  DevBuf t(ctx);
  FTN_TRY(put_table(ctx, jobs, &t.p));
  k<<<dim3((unsigned)jobs.size(), slices), 256, 0, ctx->stream>>>((const T*)t.p);
  ctx->launches += 1;
  FTN_CUDA(cudaGetLastError());
  return FTN_OK;
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
  int64_t o_px_part[2], o_py_part[2], o_gx[2], o_gy[2], o_m[2], o_tf[2], o_wk[2], o_zk[2], o_px[2], o_qy[2],
      o_ms3[2], o_rxc[2], o_ryc[2], o_sc[2];
  int64_t s_off[2];  // singular values + sweep count in the batch's shared buffer
  // Householder TSQR of the tall sides whose Gram factor is not kept:
  // chunks of qr_lx / qr_ly rows, one K x K factor slot per chunk at o_hx /
  // o_hy (slot 0 holds the result)
  int64_t o_hx[2], o_hy[2], qr_lx[2], qr_ly[2];
  // residual test of a Gram factor with dropped pivots: T (K x K) per tall
  // side at o_tx / o_ty; E = A T (rows x K) reuses the Householder slots
  int64_t o_tx[2], o_ty[2];
  int qr_px[2], qr_py[2];
  int sp_x[2], sp_y[2], rx[2], ry[2], ldx[2], ldy[2], nrot[2], mlen[2];
  int rx0[2], ry0[2];  // rows of the factors before compaction (min(rows, K))
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
    // A side is replaced by an R factor (K rows) only where that shrinks the
    // core enough to pay for the factorisation: rows beyond what the
    // compaction and the SVD take as rows (LA_MAX_DIM), or at least 5/4 K
    // rows while the partner side has more than K/8 rows (the SVD rotates
    // the shorter side, so a long side whose partner is short only lengthens
    // the rotated rows).  Any other side is its own factor (A = I A): no
    // rounding is added, and the core keeps the same nonzero singular triplets.
    // A sector that is empty on either side contributes nothing.
    auto factored = [&](int64_t rows, int64_t other) {
      if (rows <= K || other == 0) return false;
      if (rows > LA_MAX_DIM) return true;
      return 4 * rows >= 5 * K && 8 * std::min(other, K) > K;
    };
    J.tall_x[pi] = factored(R, Cc);
    J.tall_y[pi] = factored(Cc, R);
    J.rx[pi] = J.rx0[pi] = (R == 0 || Cc == 0) ? 0 : (int)(J.tall_x[pi] ? K : R);
    J.ry[pi] = J.ry0[pi] = (R == 0 || Cc == 0) ? 0 : (int)(J.tall_y[pi] ? K : Cc);
    J.o_gx[pi] = off;
    off += J.tall_x[pi] ? al(K * K) : 0;
    J.o_gy[pi] = off;
    off += J.tall_y[pi] ? al(K * K) : 0;
    // split-K over the long (row) dimension of the Gram products
    auto split_for = [&](int64_t rows) {
      const int64_t tiles = ((K + 63) / 64) * ((K + 63) / 64);
      int64_t s = std::max<int64_t>(1, (2 * (int64_t)ctx->num_sms + tiles - 1) / tiles);
      s = std::min<int64_t>(s, std::max<int64_t>(1, rows / 512));
      return (int)std::min<int64_t>(s, 64);
    };
    J.sp_x[pi] = J.tall_x[pi] ? split_for(R) : 1;
    J.sp_y[pi] = J.tall_y[pi] ? split_for(Cc) : 1;
    J.o_px_part[pi] = off;
    off += J.sp_x[pi] > 1 ? al((int64_t)J.sp_x[pi] * K * K) : 0;
    J.o_py_part[pi] = off;
    off += J.sp_y[pi] > 1 ? al((int64_t)J.sp_y[pi] * K * K) : 0;
    // Householder chunks: at least K rows (a leaf costs about as much as
    // two merges; the merge tree adds at most ~1/3 of the leaves' work), at
    // most 256 per side, a multiple of the 32-row pass
    auto chunk_rows = [&](int64_t rows) {
      int64_t L = std::max<int64_t>({K, (rows + 255) / 256, (int64_t)QR_ROWS_WIDE});
      return (L + QR_ROWS_WIDE - 1) / QR_ROWS_WIDE * QR_ROWS_WIDE;
    };
    J.qr_lx[pi] = J.tall_x[pi] ? chunk_rows(R) : 0;
    J.qr_px[pi] = J.tall_x[pi] ? (int)((R + J.qr_lx[pi] - 1) / J.qr_lx[pi]) : 0;
    J.qr_ly[pi] = J.tall_y[pi] ? chunk_rows(Cc) : 0;
    J.qr_py[pi] = J.tall_y[pi] ? (int)((Cc + J.qr_ly[pi] - 1) / J.qr_ly[pi]) : 0;
    J.o_hx[pi] = off;
    off += J.tall_x[pi] ? al(std::max<int64_t>((int64_t)J.qr_px[pi] * K * K, R * K)) : 0;
    J.o_hy[pi] = off;
    off += J.tall_y[pi] ? al(std::max<int64_t>((int64_t)J.qr_py[pi] * K * K, Cc * K)) : 0;
    J.o_tx[pi] = off;
    off += J.tall_x[pi] ? al(K * K) : 0;
    J.o_ty[pi] = off;
    off += J.tall_y[pi] ? al(K * K) : 0;
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

// Gram products of the tall sides (split over rows where that gives more
// tiles; the slabs are added by the ordered reduction) and their Cholesky jobs.
ftn_status cj_gram(CJob& J, GemmF64Batch& gb, std::vector<CholJob>& chol, int* flags, double* traces) {
  const TdPlan* P = J.P.get();
  double* ws = J.ws;
  std::vector<GemmProb> gram, reds;
  auto add_gram = [&](int K, int rows, int64_t src, int64_t ld, int64_t dst, int64_t part, int nsplit, int* flag,
                      double* trace) {
    GemmProb g = make_prob(K, K, rows, src, 1, ld, src, 1, ld);
    if (nsplit > 1) {
      g.nsplit = nsplit;
      g.kchunk = (rows + nsplit - 1) / nsplit;
      g.kchunk = (g.kchunk + 15) / 16 * 16;
      g.nsplit = (rows + g.kchunk - 1) / g.kchunk;
      gemm_plain_output(g, part, K);
      g.c_slab = (int64_t)K * K;
      // the slabs at `part`, added in split order into the plain K x K result at dst
      GemmProb r = make_prob(K, K, 0, part, 0, 0, 0, 0, 0);
      gemm_plain_output(r, dst, K);
      r.nsplit = g.nsplit;
      r.c_slab = (int64_t)K * K;
      reds.push_back(r);
    } else {
      gemm_plain_output(g, dst, K);
    }
    gram.push_back(g);
    chol.push_back({ws + dst, K, flag, trace});
  };
  for (int pi = 0; pi < 2; ++pi) {
    const int K = (int)P->K[pi];
    if (K == 0) continue;
    if (J.tall_x[pi] && P->M[pi] > 0)
      add_gram(K, (int)P->M[pi], J.o_xf + P->afoff[pi], P->ldk[pi], J.o_gx[pi], J.o_px_part[pi], J.sp_x[pi],
               flags + 2 * pi, traces + 2 * pi);
    if (J.tall_y[pi] && P->N[pi] > 0)
      add_gram(K, (int)P->N[pi], J.o_yf + P->bfoff[pi], P->ldk[pi], J.o_gy[pi], J.o_py_part[pi], J.sp_y[pi],
               flags + 2 * pi + 1, traces + 2 * pi + 1);
  }
  FTN_TRY(add_gemm_set(gb, gram, ws, ws, ws, J.ws_n, J.ws_n, J.ws_n));
  if (!red_in_bounds(reds, J.ws_n, J.ws_n)) return set_error(FTN_EINVAL, "internal error: Gram reduction out of bounds");
  add_reductions(gb, reds, ws, ws);
  return FTN_OK;
}

// Householder TSQR jobs of the tall sides selected by flags (index 2 * pi +
// side, side 0 = X, 1 = Y; bit 0), by tree level: level 0 factors
// every chunk into its own slot; level l >= 1 merges slot c + 2^(l-1) into
// slot c for every c that is a multiple of 2^l (the merged factor is upper
// triangular, its zero prefix skipped).  levels[l] receives the jobs.
void cj_qr(CJob& J, std::vector<std::vector<QrJob>>& levels, const int* flags) {
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
    if (J.tall_x[pi] && P->M[pi] > 0 && (flags[2 * pi] & 1))
      side(K, P->M[pi], J.o_xf + P->afoff[pi], P->ldk[pi], J.o_hx[pi], J.qr_lx[pi], J.qr_px[pi]);
    if (J.tall_y[pi] && P->N[pi] > 0 && (flags[2 * pi + 1] & 1))
      side(K, P->N[pi], J.o_yf + P->bfoff[pi], P->ldk[pi], J.o_hy[pi], J.qr_ly[pi], J.qr_py[pi]);
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

// ---- backward pass of the compression (ftn_compress_grad) -------------------
// Per job with cotangents and per bond-parity sector with kept states, in the
// projector form of the forward (A, B the fused sector matrices, M = R_X R_Y^T
// = U S V^T over its r singular triplets, Z = S_k^-1/2 V_k^T, W = S_k^-1/2 U_k^T):
//   X' = A R_Y^T Z^T,  Y' = W R_X B^T.
// With E_A = dX'^T A and E_B = dY' B (k x K):
//   dZ = E_A R_Y^T and dW = E_B R_X^T give dV, dU and dS (through S^-1/2);
//   dM = the thin-SVD adjoint (the rule of oracle/compress_adjoint.py) over
//        all r triplets, F_ij = 1 / (s_j^2 - s_i^2) where i or j is kept;
//   dR_X = W^T E_B + dM R_Y,  dR_Y = Z^T E_A + dM^T R_X;
//   dA = dX' Z R_Y + QR'(A, R_X, dR_X),  dB = dY'^T W R_X + QR'(B, R_Y, dR_Y),
// with QR'(A, R, dR) = A R^-1 copyltu(R dR^T) R^-T for a factored side (R
// square, full rank; no cotangent reaches Q: the projector form never forms
// it) and dR itself for a side that is its own factor; then the adjoint of
// the sign-permutes gives dX and dY.  Valid where the compression is
// differentiable (a gap at the cut, distinct nonzero singular values, full
// rank blocks); sides with dropped rows or a core with a zero singular value
// are reported as unsupported.
ftn_status cj_backward(ftn_ctx ctx, std::vector<CJob*>& gj, const std::vector<double>& sv, const double* sbuf) {
  struct Sec {
    CJob* J;
    int pi, Ma, Nb, K, ldk, rx, ry, r, ml, k;
    bool fx, fy;
    const double *A, *B, *RX, *RY, *Ms, *Tf, *Z, *W, *PA, *QB, *s;
    double tol;  // singular values at or below it (rounding level of the core) are left out
    double *dXf, *dYt, *EA, *EB, *Rot, *Oth, *Ut, *Vt, *dZ, *dW, *dRX1, *dRY1, *dUt, *dVt, *ds, *X, *Y, *inner,
        *XU, *YV, *Pt, *Qt, *T1, *SV, *dMa, *dMb, *dRX2, *dRY2, *dAd, *dBd, *RdRx, *Rix, *Hx, *Gx, *dAq, *RdRy, *Riy,
        *Hy, *Gy, *dBq;
    int *idx, *kept, *ord;
    int nord;  // rows in ord: singular values above tol, decreasing
  };
  std::vector<Sec> secs;
  std::vector<std::unique_ptr<DevBuf>> bufs;
  std::vector<double*> dAf(gj.size()), dBf(gj.size());
  for (size_t q = 0; q < gj.size(); ++q) {
    CJob& J = *gj[q];
    const TdPlan* P = J.P.get();
    std::vector<Sec> js;
    int64_t tot = P->af_elems + P->bf_elems;
    for (int pi = 0; pi < 2; ++pi) {
      if (J.k[pi] == 0) continue;
      Sec c{};
      c.J = &J;
      c.pi = pi;
      c.Ma = (int)P->M[pi], c.Nb = (int)P->N[pi], c.K = (int)P->K[pi], c.ldk = (int)P->ldk[pi];
      c.rx = J.rx[pi], c.ry = J.ry[pi], c.r = J.nrot[pi], c.ml = J.mlen[pi], c.k = J.k[pi];
      c.fx = J.tall_x[pi], c.fy = J.tall_y[pi];
      if (c.rx != J.rx0[pi] || c.ry != J.ry0[pi])
        return set_error(FTN_EUNSUPPORTED, "compression adjoint: a sector block is rank deficient (its factor has "
                                           "dropped rows)");
      const int64_t K = c.K, r = c.r, k = c.k, rx = c.rx, ry = c.ry;
      tot += c.Ma * k + k * c.Nb + 2 * k * K + r * c.ml + r * r + k * ry + k * rx + (rx + ry) * K * 3 + r * (rx + ry) +
             r + 3 * r * r + 2 * r * (rx + ry) + 2 * r * ry + 2 * rx * ry + (c.Ma + c.Nb) * K +
             (c.fx ? 4 * K * K + c.Ma * K : 0) + (c.fy ? 4 * K * K + c.Nb * K : 0) + (k + 2 * r + 2) / 2 + 8;
      js.push_back(c);
    }
    bufs.emplace_back(new DevBuf(ctx));
    bufs.back()->p = dev_alloc(ctx, (size_t)(tot + 64) * 8);
    if (!bufs.back()->p) return set_error(FTN_ENOMEM, "compression adjoint: workspace allocation failed");
    double* p = (double*)bufs.back()->p;
    dAf[q] = p;
    p += P->af_elems;
    dBf[q] = p;
    p += P->bf_elems;
    FTN_CUDA(cudaMemsetAsync(dAf[q], 0, (size_t)(P->af_elems + P->bf_elems) * 8, ctx->stream));
    for (Sec& c : js) {
      const int64_t K = c.K, r = c.r, k = c.k, rx = c.rx, ry = c.ry;
      auto take = [&](int64_t n) {
        double* x = p;
        p += n;
        return x;
      };
      c.dXf = take(c.Ma * k), c.dYt = take(k * c.Nb), c.EA = take(k * K), c.EB = take(k * K);
      c.Rot = take(r * c.ml), c.Oth = take(r * r), c.dZ = take(k * ry), c.dW = take(k * rx);
      c.dRX1 = take(rx * K), c.dRY1 = take(ry * K), c.dUt = take(r * rx), c.dVt = take(r * ry), c.ds = take(r);
      c.X = take(r * r), c.Y = take(r * r), c.inner = take(r * r), c.XU = take(r * rx), c.YV = take(r * ry);
      c.Pt = take(r * rx), c.Qt = take(r * ry), c.T1 = take(r * ry), c.SV = take(r * ry);
      c.dMa = take(rx * ry), c.dMb = take(rx * ry), c.dRX2 = take(rx * K), c.dRY2 = take(ry * K);
      c.dAd = take(c.Ma * K), c.dBd = take(c.Nb * K);
      c.RdRx = c.Rix = c.Hx = c.Gx = c.dAq = c.RdRy = c.Riy = c.Hy = c.Gy = c.dBq = nullptr;
      if (c.fx) c.RdRx = take(K * K), c.Rix = take(K * K), c.Hx = take(K * K), c.Gx = take(K * K), c.dAq = take(c.Ma * K);
      if (c.fy) c.RdRy = take(K * K), c.Riy = take(K * K), c.Hy = take(K * K), c.Gy = take(K * K), c.dBq = take(c.Nb * K);
      c.idx = reinterpret_cast<int*>(p);
      c.kept = c.idx + k;
      c.ord = c.kept + r;
      p += (k + 2 * r + 2) / 2 + 1;
      CJob& J = *c.J;
      c.A = J.ws + J.o_xf + P->afoff[c.pi];
      c.B = J.ws + J.o_yf + P->bfoff[c.pi];
      c.RX = J.ws + J.o_rxc[c.pi], c.RY = J.ws + J.o_ryc[c.pi];
      c.Ms = J.ws + J.o_m[c.pi], c.Tf = J.ws + J.o_tf[c.pi];
      c.Z = J.ws + J.o_zk[c.pi], c.W = J.ws + J.o_wk[c.pi];
      c.PA = J.ws + J.o_px[c.pi], c.QB = J.ws + J.o_qy[c.pi];
      c.s = sbuf + J.s_off[c.pi];
      // rotated rows give V (the core stored as M) or U (stored as M^T)
      c.Ut = J.trans[c.pi] ? c.Rot : c.Oth;
      c.Vt = J.trans[c.pi] ? c.Oth : c.Rot;
      // kept states in new-bond order -> Jacobi rows; kept flags per row
      std::vector<int> hk(k + 2 * r, 0);
      int j = 0;
      for (auto& cd : J.kept)
        if (cd.pi == c.pi) hk[j++] = cd.idx;
      double smax = 0.0;
      const double* sj = sv.data() + J.s_off[c.pi];
      for (int t = 0; t < r; ++t) smax = std::max(smax, sj[t]);
      c.tol = 1e-12 * smax;
      for (int t = 0; t < r; ++t)
        if (!(sj[t] > c.tol)) hk[k + t] = -1;
      for (int t = 0; t < k; ++t) hk[k + hk[t]] = 1;
      std::vector<int> ord;
      for (int t = 0; t < r; ++t)
        if (sj[t] > c.tol) ord.push_back(t);
      std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return sj[a] > sj[b]; });
      c.nord = (int)ord.size();
      std::copy(ord.begin(), ord.end(), hk.begin() + k + r);
      FTN_CUDA(cudaMemcpyAsync(c.idx, hk.data(), hk.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
      // cotangents in the fused sector coordinates: dX' rows as A's rows,
      // dY'^T columns as B's rows
      ftn_tensor gX = J.it->gXn, gY = J.it->gYn;
      const int nfa = P->nfa, nfb = P->nfb;
      for (uint32_t mA = 0; mA < (1u << nfa); ++mA) {
        if ((popc(mA) & 1) != (J.it->X->parity ^ c.pi) || P->rowsz[c.pi][mA] == 0) continue;
        const uint32_t mask = mA | ((uint32_t)c.pi << nfa);
        FTN_CUDA(cudaMemcpyAsync(c.dXf + P->rowoff[c.pi][mA] * k, (const double*)gX->data + gX->offsets[mask >> 1],
                                 (size_t)P->rowsz[c.pi][mA] * k * 8, cudaMemcpyDeviceToDevice, ctx->stream));
      }
      for (uint32_t mB = 0; mB < (1u << nfb); ++mB) {
        if ((popc(mB) & 1) != (J.it->Y->parity ^ c.pi) || P->colsz[c.pi][mB] == 0) continue;
        const uint32_t mask = (uint32_t)c.pi | (mB << 1);
        const int64_t cm = P->colsz[c.pi][mB];
        FTN_CUDA(cudaMemcpy2DAsync(c.dYt + P->coloff[c.pi][mB], (size_t)c.Nb * 8,
                                   (const double*)gY->data + gY->offsets[mask >> 1], (size_t)cm * 8, (size_t)cm * 8,
                                   (size_t)k, cudaMemcpyDeviceToDevice, ctx->stream));
      }
      secs.push_back(c);
    }
  }
  // C[m, n] = sum_k A[m, k] B[n, k] from absolute operand pointers (strides in
  // elements), row-major C with row stride ldc
  auto gemm = [&](GemmF64Batch& gb, int M, int N, int Kd, const double* a, int64_t a_sm, int64_t a_sk,
                  const double* b, int64_t b_sn, int64_t b_sk, double* cc, int64_t ldc) -> ftn_status {
    if (M <= 0 || N <= 0) return FTN_OK;
    std::vector<GemmProb> v{make_prob(M, N, Kd, 0, a_sm, a_sk, 0, b_sn, b_sk)};
    gemm_plain_output(v[0], 0, ldc);
    const int64_t an = Kd > 0 ? (int64_t)(M - 1) * a_sm + (int64_t)(Kd - 1) * a_sk + 1 : 1;
    const int64_t bn = Kd > 0 ? (int64_t)(N - 1) * b_sn + (int64_t)(Kd - 1) * b_sk + 1 : 1;
    return add_gemm_set(gb, v, a, b, cc, an, bn, (int64_t)(M - 1) * ldc + N);
  };
  auto stage = [&](auto&& body) -> ftn_status {
    GemmF64Batch gb(ctx);
    for (Sec& c : secs) FTN_TRY(body(gb, c));
    return flush_gemm_f64(gb);
  };
  // E_A = dX'^T A, E_B = dY' B; the rotated rows over their singular values
  FTN_TRY(stage([&](GemmF64Batch& gb, Sec& c) -> ftn_status {
    FTN_TRY(gemm(gb, c.k, c.K, c.Ma, c.dXf, 1, c.k, c.A, 1, c.ldk, c.EA, c.K));
    return gemm(gb, c.k, c.K, c.Nb, c.dYt, c.Nb, 1, c.B, 1, c.ldk, c.EB, c.K);
  }));
  {
    std::vector<RowDivJob> rd;
    for (Sec& c : secs) rd.push_back({c.Tf, c.Rot, c.s, c.r, c.ml, c.tol});
    FTN_TRY(launch_jobs(ctx, row_div_kernel, rd));
  }
  // the other side's vectors (stored core times the rotated ones); dZ, dW, and
  // the direct parts of dR_X, dR_Y
  FTN_TRY(stage([&](GemmF64Batch& gb, Sec& c) -> ftn_status {
    FTN_TRY(gemm(gb, c.r, c.r, c.ml, c.Rot, c.ml, 1, c.Ms, c.ml, 1, c.Oth, c.r));
    FTN_TRY(gemm(gb, c.k, c.ry, c.K, c.EA, c.K, 1, c.RY, c.K, 1, c.dZ, c.ry));
    FTN_TRY(gemm(gb, c.k, c.rx, c.K, c.EB, c.K, 1, c.RX, c.K, 1, c.dW, c.rx));
    FTN_TRY(gemm(gb, c.ry, c.K, c.k, c.Z, 1, c.ry, c.EA, 1, c.K, c.dRY1, c.K));
    return gemm(gb, c.rx, c.K, c.k, c.W, 1, c.rx, c.EB, 1, c.K, c.dRX1, c.K);
  }));
  {
    std::vector<RowDivJob> rd;
    for (Sec& c : secs) rd.push_back({c.Oth, c.Oth, c.s, c.r, c.r, c.tol});
    FTN_TRY(launch_jobs(ctx, row_div_kernel, rd));
  }
  // The rebuilt vectors (rows of Oth, each of length r) re-orthonormalised in
  // the order of decreasing singular values (Gram-Schmidt order: the vectors
  // of the larger singular values, the more accurate ones, first).  Blocks of
  // ORTH_B rows of the ordered copy Vo: a block is projected twice against
  // every row before it (H = V_prev V_b^T, V_b -= H^T V_prev), then made
  // orthonormal within itself by CholeskyQR (G = V_b V_b^T = L L^T, V_b :=
  // L^{-1} V_b), which the near-orthonormal rows keep stable.  In exact
  // arithmetic this is the QR factorisation's Q, as Gram-Schmidt gives it;
  // the products run as grouped FP64 GEMMs across the GPU.
  {
    struct Orth {
      double *Vo, *H, *T, *G;
    };
    std::vector<Orth> ow(secs.size());
    std::vector<std::unique_ptr<DevBuf>> obufs;
    std::vector<RowsJob> mv;
    int nblk = 0;
    for (size_t q = 0; q < secs.size(); ++q) {
      const Sec& c = secs[q];
      if (c.nord == 0 || c.r == 0) continue;
      const int64_t nr = c.nord, r = c.r;
      obufs.emplace_back(new DevBuf(ctx));
      obufs.back()->p = dev_alloc(ctx, (size_t)(nr * r + nr * ORTH_B + ORTH_B * r + ORTH_B * ORTH_B + 16) * 8);
      if (!obufs.back()->p) return set_error(FTN_ENOMEM, "compression adjoint: workspace allocation failed");
      double* p = (double*)obufs.back()->p;
      ow[q] = {p, p + nr * r, p + nr * r + nr * ORTH_B, p + nr * r + nr * ORTH_B + ORTH_B * r};
      mv.push_back({c.Oth, ow[q].Vo, c.ord, c.nord, c.r, 0});
      nblk = std::max(nblk, (c.nord + ORTH_B - 1) / ORTH_B);
    }
    FTN_TRY(launch_jobs(ctx, rows_move_kernel, mv));
    for (int bk = 0; bk < nblk; ++bk) {
      const int prev = bk * ORTH_B;
      auto in_blk = [&](const Sec& c) { return c.r > 0 && prev < c.nord; };
      auto nb_of = [&](const Sec& c) { return std::min(ORTH_B, c.nord - prev); };
      for (int pass = 0; pass < 2 && prev > 0; ++pass) {
        FTN_TRY(stage([&](GemmF64Batch& gb, Sec& c) -> ftn_status {
          if (!in_blk(c)) return FTN_OK;
          const Orth& o = ow[&c - secs.data()];
          const double* Vb = o.Vo + (int64_t)prev * c.r;
          return gemm(gb, prev, nb_of(c), c.r, o.Vo, c.r, 1, Vb, c.r, 1, o.H, nb_of(c));
        }));
        FTN_TRY(stage([&](GemmF64Batch& gb, Sec& c) -> ftn_status {
          if (!in_blk(c)) return FTN_OK;
          const Orth& o = ow[&c - secs.data()];
          return gemm(gb, nb_of(c), c.r, prev, o.H, 1, nb_of(c), o.Vo, 1, c.r, o.T, c.r);
        }));
        std::vector<AxpyJob> sub;
        for (Sec& c : secs)
          if (in_blk(c)) {
            double* Vb = ow[&c - secs.data()].Vo + (int64_t)prev * c.r;
            sub.push_back({Vb, ow[&c - secs.data()].T, Vb, nullptr, nullptr, (int64_t)nb_of(c) * c.r, c.r, -1.0});
          }
        FTN_TRY(launch_jobs(ctx, axpy_kernel, sub));
      }
      FTN_TRY(stage([&](GemmF64Batch& gb, Sec& c) -> ftn_status {
        if (!in_blk(c)) return FTN_OK;
        const Orth& o = ow[&c - secs.data()];
        const double* Vb = o.Vo + (int64_t)prev * c.r;
        return gemm(gb, nb_of(c), nb_of(c), c.r, Vb, c.r, 1, Vb, c.r, 1, o.G, nb_of(c));
      }));
      std::vector<CholInvJob> ci;
      for (Sec& c : secs)
        if (in_blk(c)) ci.push_back({ow[&c - secs.data()].G, nb_of(c)});
      FTN_TRY(launch_jobs(ctx, chol_inv_small_kernel, ci));
      FTN_TRY(stage([&](GemmF64Batch& gb, Sec& c) -> ftn_status {
        if (!in_blk(c)) return FTN_OK;
        const Orth& o = ow[&c - secs.data()];
        const double* Vb = o.Vo + (int64_t)prev * c.r;
        return gemm(gb, nb_of(c), c.r, nb_of(c), o.G, nb_of(c), 1, Vb, 1, c.r, o.T, c.r);
      }));
      std::vector<AxpyJob> cp;
      for (Sec& c : secs)
        if (in_blk(c)) {
          double* Vb = ow[&c - secs.data()].Vo + (int64_t)prev * c.r;
          cp.push_back({nullptr, ow[&c - secs.data()].T, Vb, nullptr, nullptr, (int64_t)nb_of(c) * c.r, c.r, 1.0});
        }
      FTN_TRY(launch_jobs(ctx, axpy_kernel, cp));
    }
    std::vector<RowsJob> back;
    for (size_t q = 0; q < secs.size(); ++q)
      if (secs[q].nord > 0 && secs[q].r > 0)
        back.push_back({ow[q].Vo, secs[q].Oth, secs[q].ord, secs[q].nord, secs[q].r, 1});
    FTN_TRY(launch_jobs(ctx, rows_move_kernel, back));
  }
  {
    std::vector<CotJob> cj;
    for (Sec& c : secs) cj.push_back({c.dZ, c.dW, c.Ut, c.Vt, c.s, c.idx, c.dUt, c.dVt, c.ds, c.k, c.r, c.rx, c.ry});
    FTN_TRY(launch_jobs(ctx, svd_cot_kernel, cj));
  }
  // X = U^T dU, Y = V^T dV, then X^T Ut and Y^T Vt
  FTN_TRY(stage([&](GemmF64Batch& gb, Sec& c) -> ftn_status {
    FTN_TRY(gemm(gb, c.r, c.r, c.rx, c.Ut, c.rx, 1, c.dUt, c.rx, 1, c.X, c.r));
    return gemm(gb, c.r, c.r, c.ry, c.Vt, c.ry, 1, c.dVt, c.ry, 1, c.Y, c.r);
  }));
  FTN_TRY(stage([&](GemmF64Batch& gb, Sec& c) -> ftn_status {
    FTN_TRY(gemm(gb, c.r, c.rx, c.r, c.X, 1, c.r, c.Ut, 1, c.rx, c.XU, c.rx));
    return gemm(gb, c.r, c.ry, c.r, c.Y, 1, c.r, c.Vt, 1, c.ry, c.YV, c.ry);
  }));
  {
    std::vector<InnerJob> ij;
    std::vector<AxpyJob> ax;
    for (Sec& c : secs) {
      ij.push_back({c.X, c.Y, c.s, c.ds, c.kept, c.inner, c.r});
      ax.push_back({c.dUt, c.XU, c.Pt, nullptr, nullptr, (int64_t)c.r * c.rx, c.rx, -1.0});  // (I - U U^T) dU
      ax.push_back({c.dVt, c.YV, c.Qt, nullptr, nullptr, (int64_t)c.r * c.ry, c.ry, -1.0});  // (I - V V^T) dV
    }
    FTN_TRY(launch_jobs(ctx, svd_inner_kernel, ij));
    FTN_TRY(launch_jobs(ctx, axpy_kernel, ax));
  }
  FTN_TRY(stage([&](GemmF64Batch& gb, Sec& c) -> ftn_status {
    return gemm(gb, c.r, c.ry, c.r, c.inner, c.r, 1, c.Vt, 1, c.ry, c.T1, c.ry);
  }));
  {
    std::vector<AxpyJob> ax;
    for (Sec& c : secs) {
      ax.push_back({c.T1, c.Qt, c.T1, c.s, c.kept, (int64_t)c.r * c.ry, c.ry, 1.0});     // inner V^T + S^-1 dV^T (I - V V^T)
      ax.push_back({nullptr, c.Vt, c.SV, c.s, c.kept, (int64_t)c.r * c.ry, c.ry, 1.0});  // S^-1 V^T
    }
    FTN_TRY(launch_jobs(ctx, axpy_kernel, ax));
  }
  // dM = U (inner V^T + S^-1 dV^T (I - V V^T)) + (I - U U^T) dU S^-1 V^T
  FTN_TRY(stage([&](GemmF64Batch& gb, Sec& c) -> ftn_status {
    FTN_TRY(gemm(gb, c.rx, c.ry, c.r, c.Ut, 1, c.rx, c.T1, 1, c.ry, c.dMa, c.ry));
    return gemm(gb, c.rx, c.ry, c.r, c.Pt, 1, c.rx, c.SV, 1, c.ry, c.dMb, c.ry);
  }));
  {
    std::vector<AxpyJob> ax;
    for (Sec& c : secs) ax.push_back({c.dMa, c.dMb, c.dMa, nullptr, nullptr, (int64_t)c.rx * c.ry, c.ry, 1.0});
    FTN_TRY(launch_jobs(ctx, axpy_kernel, ax));
  }
  // dR_X = W^T E_B + dM R_Y, dR_Y = Z^T E_A + dM^T R_X
  FTN_TRY(stage([&](GemmF64Batch& gb, Sec& c) -> ftn_status {
    FTN_TRY(gemm(gb, c.rx, c.K, c.ry, c.dMa, c.ry, 1, c.RY, 1, c.K, c.dRX2, c.K));
    return gemm(gb, c.ry, c.K, c.rx, c.dMa, 1, c.ry, c.RX, 1, c.K, c.dRY2, c.K);
  }));
  {
    std::vector<AxpyJob> ax;
    for (Sec& c : secs) {
      ax.push_back({c.dRX1, c.dRX2, c.dRX1, nullptr, nullptr, (int64_t)c.rx * c.K, c.K, 1.0});
      ax.push_back({c.dRY1, c.dRY2, c.dRY1, nullptr, nullptr, (int64_t)c.ry * c.K, c.K, 1.0});
    }
    FTN_TRY(launch_jobs(ctx, axpy_kernel, ax));
  }
  // factored sides: R dR^T, R^-1
  FTN_TRY(stage([&](GemmF64Batch& gb, Sec& c) -> ftn_status {
    if (c.fx) FTN_TRY(gemm(gb, c.K, c.K, c.K, c.RX, c.K, 1, c.dRX1, c.K, 1, c.RdRx, c.K));
    if (c.fy) FTN_TRY(gemm(gb, c.K, c.K, c.K, c.RY, c.K, 1, c.dRY1, c.K, 1, c.RdRy, c.K));
    return FTN_OK;
  }));
  {
    std::vector<SqJob> cl, ti;
    for (Sec& c : secs) {
      if (c.fx) cl.push_back({c.RdRx, nullptr, c.K}), ti.push_back({c.Rix, c.RX, c.K});
      if (c.fy) cl.push_back({c.RdRy, nullptr, c.K}), ti.push_back({c.Riy, c.RY, c.K});
    }
    FTN_TRY(launch_jobs(ctx, copyltu_kernel, cl));
    FTN_TRY(launch_jobs(ctx, tri_inverse_kernel, ti));
  }
  // H = R^-1 copyltu(R dR^T), G = H R^-T, then A G
  FTN_TRY(stage([&](GemmF64Batch& gb, Sec& c) -> ftn_status {
    if (c.fx) FTN_TRY(gemm(gb, c.K, c.K, c.K, c.Rix, c.K, 1, c.RdRx, 1, c.K, c.Hx, c.K));
    if (c.fy) FTN_TRY(gemm(gb, c.K, c.K, c.K, c.Riy, c.K, 1, c.RdRy, 1, c.K, c.Hy, c.K));
    return FTN_OK;
  }));
  FTN_TRY(stage([&](GemmF64Batch& gb, Sec& c) -> ftn_status {
    if (c.fx) FTN_TRY(gemm(gb, c.K, c.K, c.K, c.Hx, c.K, 1, c.Rix, c.K, 1, c.Gx, c.K));
    if (c.fy) FTN_TRY(gemm(gb, c.K, c.K, c.K, c.Hy, c.K, 1, c.Riy, c.K, 1, c.Gy, c.K));
    return FTN_OK;
  }));
  // A G (factored) and the direct parts dX' P_X^T, dY'^T Q_Y^T
  FTN_TRY(stage([&](GemmF64Batch& gb, Sec& c) -> ftn_status {
    if (c.fx) FTN_TRY(gemm(gb, c.Ma, c.K, c.K, c.A, c.ldk, 1, c.Gx, 1, c.K, c.dAq, c.K));
    if (c.fy) FTN_TRY(gemm(gb, c.Nb, c.K, c.K, c.B, c.ldk, 1, c.Gy, 1, c.K, c.dBq, c.K));
    FTN_TRY(gemm(gb, c.Ma, c.K, c.k, c.dXf, c.k, 1, c.PA, 1, c.K, c.dAd, c.K));
    return gemm(gb, c.Nb, c.K, c.k, c.dYt, 1, c.Nb, c.QB, 1, c.K, c.dBd, c.K);
  }));
  {
    std::vector<Add2Job> ad;
    for (Sec& c : secs) {
      const TdPlan* P = c.J->P.get();
      const size_t q = std::find(gj.begin(), gj.end(), c.J) - gj.begin();
      double* da = dAf[q] + P->afoff[c.pi];
      double* db = dBf[q] + P->bfoff[c.pi];
      ad.push_back({c.dAd, da, c.Ma, c.K, c.K, c.ldk});
      ad.push_back({c.fx ? c.dAq : c.dRX1, da, c.Ma, c.K, c.K, c.ldk});  // a side that is its own factor: rx = Ma
      ad.push_back({c.dBd, db, c.Nb, c.K, c.K, c.ldk});
      ad.push_back({c.fy ? c.dBq : c.dRY1, db, c.Nb, c.K, c.K, c.ldk});
    }
    // the four adds of a sector touch the same rows: one launch each, in order
    for (int w = 0; w < 4; ++w) {
      std::vector<Add2Job> one;
      for (size_t i = w; i < ad.size(); i += 4) one.push_back(ad[i]);
      FTN_TRY(launch_jobs(ctx, add2_kernel, one, 32));
    }
  }
  // dX, dY: the adjoint of the forward's sign-permutes
  for (size_t q = 0; q < gj.size(); ++q) {
    CJob& J = *gj[q];
    const TdPlan* P = J.P.get();
    ftn_tensor X = J.it->X, Y = J.it->Y;
    int32_t xd0[MAXR], xd1[MAXR], yd0[MAXR], yd1[MAXR];
    for (int l = 0; l < X->rank; ++l) xd0[l] = X->d0[l], xd1[l] = X->d1[l];
    for (int l = 0; l < Y->rank; ++l) yd0[l] = Y->d0[l], yd1[l] = Y->d1[l];
    FTN_TRY(make_tensor(ctx, X->rank, xd0, xd1, X->dual, X->parity, FTN_F64, &J.it->dX));
    FTN_TRY(make_tensor(ctx, Y->rank, yd0, yd1, Y->dual, Y->parity, FTN_F64, &J.it->dY));
    FTN_CUDA(cudaMemsetAsync(J.it->dX->data, 0, (size_t)J.it->dX->numel * 8, ctx->stream));
    FTN_CUDA(cudaMemsetAsync(J.it->dY->data, 0, (size_t)J.it->dY->numel * 8, ctx->stream));
    for (int side = 0; side < 2; ++side) {
      const std::vector<PermJob>& jb = side ? P->jb : P->ja;
      if (jb.empty()) continue;
      DevBuf t(ctx);
      FTN_TRY(put_table(ctx, jb, &t.p));
      perm_adjoint_kernel<<<(unsigned)jb.size(), 256, 0, ctx->stream>>>(
          (const PermJob*)t.p, side ? dBf[q] : dAf[q], (double*)(side ? J.it->dY->data : J.it->dX->data));
      ctx->launches += 1;
      FTN_CUDA(cudaGetLastError());
    }
  }
  return FTN_OK;
}

}  // namespace

// A compression's forward kept for its adjoint: the item (inputs, bond, chi),
// its job (plan, offsets into the workspace, kept states), the workspace it
// ran in, and the singular values it read back.
struct CompressState {
  ftn_ctx ctx = nullptr;
  CompressItem item;
  std::vector<CJob> jobs;
  void* buf = nullptr;
  std::vector<double> sv;
  double* sbuf = nullptr;
  int64_t xn_numel = 0, yn_numel = 0;
  int xn_parity = 0, yn_parity = 0;
};

// Batched compression: every stage of every job contributes to one launch
// per kernel; two host synchronisations per batch (the R-factor row counts
// and the singular values).
ftn_status compress_batch(ftn_ctx ctx, std::vector<CompressItem>& items) {
  if (!ctx) return set_error(FTN_EINVAL, "null argument");
  if (items.empty()) return FTN_OK;
  if (stream_capturing(ctx->stream))  // the kept dimensions are read back to the host
    return set_error(FTN_EUNSUPPORTED, "compression cannot run while the stream is captured into a graph");
  std::vector<CJob> jobs(items.size());
  int64_t total = 0;
  for (size_t i = 0; i < items.size(); ++i) {
    jobs[i].it = &items[i];
    FTN_TRY(cj_prepare(ctx, jobs[i]));
    jobs[i].ws_off = total;
    total += jobs[i].ws_n;
  }
  // shared small buffers after the jobs' workspaces: [row counts and
  // Cholesky flags: 8 ints per job | singular values]
  int64_t s_total = 0;
  for (CJob& J : jobs)
    for (int pi = 0; pi < 2; ++pi) {
      J.s_off[pi] = s_total;
      s_total += J.nrot[pi] + 1;  // values, then the sweep count
    }
  const int64_t cnt_words = ((int64_t)jobs.size() * 8 * (int64_t)sizeof(int) + 7) / 8;
  const int64_t chk_words = (int64_t)jobs.size() * 8;  // per job: |A|_F^2 of the 4 sides, then |E|_F^2
  // a kept forward (batch of one, inputs kept, no cotangents) gets a
  // workspace of its own, handed to the state at the end
  const bool keep = items.size() == 1 && items[0].keep_state && items[0].keep_inputs && !items[0].gXn &&
                    !items[0].gYn;
  const ftn_tensor in_x = items[0].X, in_y = items[0].Y;
  DevBuf own(ctx);
  const size_t ws_bytes = (size_t)(total + cnt_words + chk_words + s_total + 32) * 8;
  if (keep) own.p = dev_alloc(ctx, ws_bytes);
  double* ws = keep ? (double*)own.p : (double*)workspace(ctx, ws_bytes);
  if (!ws) return set_error(FTN_ENOMEM, "workspace allocation failed");
  for (CJob& J : jobs) J.ws = ws + J.ws_off;
  int* cnt = (int*)(ws + total);
  double* chk = ws + total + cnt_words;
  double* sbuf = ws + total + cnt_words + chk_words;

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
  // ---- 2. R factors: Gram matrices and semi-definite Cholesky (flags unresolved sides) ----
  // per job: cnt[8q + 2 pi + side] = nonzero rows of the factor, cnt[8q + 4 + 2 pi + side] = flag
  FTN_CUDA(cudaMemsetAsync(cnt, 0, jobs.size() * 8 * sizeof(int), ctx->stream));
  {
    GemmF64Batch gb(ctx);
    std::vector<CholJob> chol;
    for (size_t q = 0; q < jobs.size(); ++q) FTN_TRY(cj_gram(jobs[q], gb, chol, cnt + 8 * q + 4, chk + 8 * q));
    FTN_TRY(flush_gemm_f64(gb));
    if (!chol.empty()) {
      DevBuf t_chol(ctx);
      FTN_TRY(put_table(ctx, chol, &t_chol.p));
      const int rec = prof_begin(ctx, "cholesky", 0, 0);
      chol_kernel<<<(unsigned)chol.size(), LA_THREADS, 0, ctx->stream>>>((const CholJob*)t_chol.p);
      ctx->launches += 1;
      FTN_CUDA(cudaGetLastError());
      prof_end(ctx, rec);
    }
  }
  // ---- 2b. nonzero rows of the R factors (one synchronisation for the counts
  //      and flags).  Sides with an unresolved pivot are factored again by
  //      Householder TSQR (one launch per tree level) and compacted again.  The
  //      residual test of the sides with dropped pivots is launched here and
  //      read back with the singular values, the Gram factor used meanwhile; a
  //      side that fails it is factored by TSQR and its job's cores decomposed
  //      again. ----
  std::vector<int> hc(8 * jobs.size(), 0);
  // sel[4 q + 2 pi + side] != 0 selects a side (side 0 = X, 1 = Y)
  auto compact = [&](const std::vector<int>& sel) -> ftn_status {
    std::vector<CompactJob> cj;
    for (size_t q = 0; q < jobs.size(); ++q) {
      CJob& J = jobs[q];
      for (int pi = 0; pi < 2; ++pi) {
        const int K = (int)J.P->K[pi];
        if (K == 0 || J.rx0[pi] == 0 || J.ry0[pi] == 0) continue;
        if (sel[4 * q + 2 * pi])
          cj.push_back({J.ws + J.rx_off[pi], J.ws + J.o_rxc[pi], cnt + 8 * q + 2 * pi, J.rx0[pi], K, J.ldx[pi]});
        if (sel[4 * q + 2 * pi + 1])
          cj.push_back({J.ws + J.ry_off[pi], J.ws + J.o_ryc[pi], cnt + 8 * q + 2 * pi + 1, J.ry0[pi], K, J.ldy[pi]});
      }
    }
    if (!cj.empty()) {
      DevBuf t_cj(ctx);
      FTN_TRY(put_table(ctx, cj, &t_cj.p));
      compact_rows_kernel<<<(unsigned)cj.size(), 256, 0, ctx->stream>>>((const CompactJob*)t_cj.p);
      ctx->launches += 1;
      FTN_CUDA(cudaGetLastError());
    }
    FTN_CUDA(cudaMemcpyAsync(hc.data(), cnt, hc.size() * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    FTN_CUDA(cudaStreamSynchronize(ctx->stream));
    return FTN_OK;
  };
  // Householder TSQR of the selected (tall) sides into their slots, then their
  // compaction (profile label: the unresolved band's, or the failed residual's)
  auto tsqr = [&](const std::vector<int>& sel, const char* label) -> ftn_status {
    std::vector<std::vector<QrJob>> levels;
    for (size_t q = 0; q < jobs.size(); ++q) cj_qr(jobs[q], levels, sel.data() + 4 * q);
    if (levels.empty()) return FTN_OK;
    FTN_TRY(setup_qr_kernels());
    for (auto& lv : levels) {
      // three variants by bond width (one launch each): factor in shared
      // memory, 32-row passes, 16-row passes
      std::vector<QrJob> part[3];
      for (const QrJob& qj : lv) part[qj.K <= QR_RSMEM_K ? 0 : qj.K <= QR_WIDE_K ? 1 : 2].push_back(qj);
      for (int v = 0; v < 3; ++v) {
        if (part[v].empty()) continue;
        int kmax = 0;
        for (const QrJob& qj : part[v]) kmax = std::max(kmax, qj.K);
        DevBuf t_qr(ctx);
        FTN_TRY(put_table(ctx, part[v], &t_qr.p));
        const int rec = prof_begin(ctx, label, 0, 0);
        const unsigned g = (unsigned)part[v].size();
        const QrJob* tj = (const QrJob*)t_qr.p;
        if (v == 0)
          qr_stream_kernel<QR_ROWS_WIDE, true><<<g, QR_THREADS, ((size_t)kmax * kmax + QR_ROWS_WIDE * kmax) * 8,
                                                ctx->stream>>>(tj);
        else if (v == 1)
          qr_stream_kernel<QR_ROWS_WIDE, false><<<g, QR_THREADS, (size_t)QR_ROWS_WIDE * kmax * 8, ctx->stream>>>(tj);
        else
          qr_stream_kernel<QR_ROWS, false><<<g, QR_THREADS, (size_t)QR_ROWS * kmax * 8, ctx->stream>>>(tj);
        ctx->launches += 1;
        FTN_CUDA(cudaGetLastError());
        prof_end(ctx, rec);
      }
    }
    for (size_t q = 0; q < jobs.size(); ++q) {
      CJob& J = jobs[q];
      for (int pi = 0; pi < 2; ++pi) {
        const int K = (int)J.P->K[pi];
        if (sel[4 * q + 2 * pi]) J.rx_off[pi] = J.o_hx[pi], J.ldx[pi] = K;
        if (sel[4 * q + 2 * pi + 1]) J.ry_off[pi] = J.o_hy[pi], J.ldy[pi] = K;
      }
    }
    return compact(sel);
  };
  // shapes of a job's cores from the row counts of its compacted factors
  auto counts = [&](size_t q) -> ftn_status {
    CJob& J = jobs[q];
    for (int pi = 0; pi < 2; ++pi) J.rx[pi] = J.rx0[pi], J.ry[pi] = J.ry0[pi];
    const int c4[4] = {hc[8 * q], hc[8 * q + 1], hc[8 * q + 2], hc[8 * q + 3]};
    return cj_counts(J, c4);
  };
  FTN_TRY(compact(std::vector<int>(4 * jobs.size(), 1)));
  {
    std::vector<int> band(4 * jobs.size(), 0);
    for (size_t q = 0; q < jobs.size(); ++q)
      for (int k = 0; k < 4; ++k) band[4 * q + k] = hc[8 * q + 4 + k] & 1;
    FTN_TRY(tsqr(band, "householder_qr"));
  }
  bool residual_pending = false;
  {
    std::vector<ResidTJob> rt[2];  // by variant: R^T in shared memory, in global memory
    std::vector<SumSqJob> sq;
    GemmF64Batch gb(ctx);
    int kmax_sm = 0;
    for (size_t q = 0; q < jobs.size(); ++q) {
      CJob& J = jobs[q];
      std::vector<GemmProb> eg;
      for (int pi = 0; pi < 2; ++pi)
        for (int side = 0; side < 2; ++side) {
          if (hc[8 * q + 4 + 2 * pi + side] != 2) continue;  // dropped pivots only, none unresolved
          const int K = (int)J.P->K[pi];
          const int64_t rows = side ? J.P->N[pi] : J.P->M[pi];
          const int64_t src = side ? J.o_yf + J.P->bfoff[pi] : J.o_xf + J.P->afoff[pi];
          const int64_t rf = side ? J.o_gy[pi] : J.o_gx[pi], tf = side ? J.o_ty[pi] : J.o_tx[pi];
          const int64_t ef = side ? J.o_hy[pi] : J.o_hx[pi];
          const int v = K <= RESID_SMEM_K ? 0 : 1;
          if (!v) kmax_sm = std::max(kmax_sm, K);
          for (int c0 = 0; c0 < K; c0 += 32) rt[v].push_back({J.ws + rf, J.ws + tf, K, c0});
          GemmProb g = make_prob((int)rows, K, K, src, J.P->ldk[pi], 1, tf, 1, K);
          gemm_plain_output(g, ef, K);
          eg.push_back(g);
          sq.push_back({J.ws + ef, rows * K, chk + 8 * q + 4 + 2 * pi + side});
        }
      if (!eg.empty()) FTN_TRY(add_gemm_set(gb, eg, J.ws, J.ws, J.ws, J.ws_n, J.ws_n, J.ws_n));
    }
    if (!sq.empty()) {
      FTN_TRY(setup_qr_kernels());
      for (int v = 0; v < 2; ++v) {
        if (rt[v].empty()) continue;
        DevBuf t_rt(ctx);
        FTN_TRY(put_table(ctx, rt[v], &t_rt.p));
        if (v == 0)
          dropped_residual_kernel<true><<<(unsigned)rt[0].size(), 128,
                                          ((size_t)kmax_sm * kmax_sm + 5 * (size_t)kmax_sm) * 8, ctx->stream>>>(
              (const ResidTJob*)t_rt.p);
        else
          dropped_residual_kernel<false><<<(unsigned)rt[1].size(), 128, 0, ctx->stream>>>((const ResidTJob*)t_rt.p);
        ctx->launches += 1;
        FTN_CUDA(cudaGetLastError());
      }
      FTN_TRY(flush_gemm_f64(gb));
      DevBuf t_sq(ctx);
      FTN_TRY(put_table(ctx, sq, &t_sq.p));
      sumsq_kernel<<<(unsigned)sq.size(), 256, 0, ctx->stream>>>((const SumSqJob*)t_sq.p);
      ctx->launches += 1;
      FTN_CUDA(cudaGetLastError());
      residual_pending = true;
    }
  }
  for (size_t q = 0; q < jobs.size(); ++q) FTN_TRY(counts(q));
  // ---- 3. core M = R_X R_Y^T (stored with the rotated side as rows) and SVD ----
  auto core_svd = [&](const std::vector<size_t>& which) -> ftn_status {
    GemmF64Batch gb(ctx);
    std::vector<SvdJob> svd;
    for (size_t q : which) {
      CJob& J = jobs[q];
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
        double* sp = sbuf + J.s_off[pi];
        svd.push_back({J.ws + J.o_m[pi], J.ws + J.o_tf[pi], sp, (int*)(sp + J.nrot[pi]), J.nrot[pi], J.mlen[pi]});
      }
      FTN_TRY(add_gemm_set(gb, mg, J.ws, J.ws, J.ws, J.ws_n, J.ws_n, J.ws_n));
    }
    FTN_TRY(flush_gemm_f64(gb));
    if (svd.empty()) return FTN_OK;
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
    return FTN_OK;
  };
  {
    std::vector<size_t> every(jobs.size());
    for (size_t q = 0; q < jobs.size(); ++q) every[q] = q;
    FTN_TRY(core_svd(every));
  }
  std::vector<double> sv_host;  // singular values (Jacobi order) and sweep counts, kept for the adjoint
  // ---- 4. pooled truncation (one synchronisation for the singular values and
  //      the residual norms; a second only when a residual test failed) ----
  {
    std::vector<double>& sv = sv_host;
    sv.assign(s_total + 1, 0.0);
    std::vector<double> hk(chk_words);
    if (s_total) FTN_CUDA(cudaMemcpyAsync(sv.data(), sbuf, s_total * 8, cudaMemcpyDeviceToHost, ctx->stream));
    if (residual_pending)
      FTN_CUDA(cudaMemcpyAsync(hk.data(), chk, chk_words * 8, cudaMemcpyDeviceToHost, ctx->stream));
    FTN_CUDA(cudaStreamSynchronize(ctx->stream));
    if (residual_pending) {
      // the Gram factor stands when the dropped columns are within 1e-12 of the kept span
      std::vector<int> fail(4 * jobs.size(), 0);
      std::vector<size_t> redo;
      for (size_t q = 0; q < jobs.size(); ++q) {
        bool any = false;
        for (int k = 0; k < 4; ++k)
          if (hc[8 * q + 4 + k] == 2 && !(hk[8 * q + 4 + k] <= 1e-24 * hk[8 * q + k])) fail[4 * q + k] = 1, any = true;
        if (any) redo.push_back(q);
      }
      if (!redo.empty()) {
        FTN_TRY(tsqr(fail, "householder_qr_redo"));
        for (size_t q : redo) FTN_TRY(counts(q));
        FTN_TRY(core_svd(redo));
        if (s_total) FTN_CUDA(cudaMemcpyAsync(sv.data(), sbuf, s_total * 8, cudaMemcpyDeviceToHost, ctx->stream));
        FTN_CUDA(cudaStreamSynchronize(ctx->stream));
      }
    }
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
    // (needed where a kept singular value is small: the error of q_j is about
    // m eps s_max / s_j, below 1e-11 once every kept s_j >= 1e-2 s_max)
    std::vector<OrthJob> orth;
    for (CJob& J : jobs)
      for (int pi = 0; pi < 2; ++pi) {
        if (J.k[pi] < 2) continue;
        double smin = J.kept.front().s;
        for (auto& c : J.kept)
          if (c.pi == pi) smin = std::min(smin, c.s);
        if (smin < 1e-2 * J.kept.front().s)
          orth.push_back({J.ws + (J.trans[pi] ? J.o_zk[pi] : J.o_wk[pi]), J.ws + J.o_sc[pi], J.k[pi], J.nrot[pi]});
      }
    if (!orth.empty()) {
      DevBuf t_orth(ctx);
      FTN_TRY(put_table(ctx, orth, &t_orth.p));
      const int rec = prof_begin(ctx, "orth_nside", 0, 0);
      orth_rows_kernel<<<(unsigned)orth.size(), 256, 0, ctx->stream>>>((const OrthJob*)t_orth.p);
      ctx->launches += 1;
      FTN_CUDA(cudaGetLastError());
      prof_end(ctx, rec);
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
  // ---- 6. adjoint, for the items that carry cotangents of the new pair ----
  {
    std::vector<CJob*> gj;
    for (CJob& J : jobs) {
      if (!J.it->gXn && !J.it->gYn) continue;
      const ftn_tensor g[2] = {J.it->gXn, J.it->gYn}, t[2] = {J.Xn, J.Yn};
      for (int w = 0; w < 2; ++w) {
        bool ok = g[w] && g[w]->dtype == FTN_F64 && g[w]->rank == t[w]->rank && g[w]->parity == t[w]->parity;
        for (int l = 0; ok && l < t[w]->rank; ++l)
          ok = g[w]->d0[l] == t[w]->d0[l] && g[w]->d1[l] == t[w]->d1[l] && g[w]->dual[l] == t[w]->dual[l];
        if (!ok)
          return set_error(FTN_ESHAPE, "compression adjoint: a cotangent does not have the legs, parity and FP64 "
                                       "type of the compressed tensor");
      }
      gj.push_back(&J);
    }
    if (!gj.empty()) FTN_TRY(cj_backward(ctx, gj, sv_host, sbuf));
  }
  outs.ok = true;
  for (CJob& J : jobs) {
    if (J.it->gXn || J.it->gYn) {  // the adjoint keeps the inputs; the forward pair was only needed here
      ftn_tensor_free(J.Xn);
      ftn_tensor_free(J.Yn);
      continue;
    }
    if (!J.it->keep_inputs) {
      ftn_tensor_free(J.it->X);
      ftn_tensor_free(J.it->Y);
    }
    J.it->X = J.Xn;
    J.it->Y = J.Yn;
  }
  if (keep) {
    CompressState* st = new CompressState;
    st->ctx = ctx;
    st->item = items[0];
    st->item.X = in_x;
    st->item.Y = in_y;
    st->item.keep_state = nullptr;
    st->item.info = nullptr;
    st->xn_numel = jobs[0].Xn->numel, st->yn_numel = jobs[0].Yn->numel;
    st->xn_parity = jobs[0].Xn->parity, st->yn_parity = jobs[0].Yn->parity;
    st->jobs = std::move(jobs);
    st->jobs[0].it = &st->item;
    st->jobs[0].Xn = st->jobs[0].Yn = nullptr;  // the compressed pair belongs to the caller
    st->buf = own.p;
    own.p = nullptr;
    st->sv = sv_host;
    st->sbuf = sbuf;
    *items[0].keep_state = st;
  }
  return FTN_OK;
}

ftn_status compress_backward(ftn_ctx ctx, CompressState* st, ftn_tensor gXn, ftn_tensor gYn, ftn_tensor* dX,
                             ftn_tensor* dY) {
  if (!ctx || !st || !gXn || !gYn || !dX || !dY) return set_error(FTN_EINVAL, "null argument");
  if (st->ctx != ctx) return set_error(FTN_EINVAL, "compression adjoint: state of another context");
  if (gXn->dtype != FTN_F64 || gYn->dtype != FTN_F64 || gXn->numel != st->xn_numel || gYn->numel != st->yn_numel ||
      gXn->parity != st->xn_parity || gYn->parity != st->yn_parity)
    return set_error(FTN_ESHAPE, "compression adjoint: a cotangent does not match the compressed pair");
  st->item.gXn = gXn;
  st->item.gYn = gYn;
  st->item.dX = st->item.dY = nullptr;
  std::vector<CJob*> gj{&st->jobs[0]};
  const ftn_status s = cj_backward(ctx, gj, st->sv, st->sbuf);
  st->item.gXn = st->item.gYn = nullptr;
  if (s != FTN_OK) {
    ftn_tensor_free(st->item.dX);
    ftn_tensor_free(st->item.dY);
    st->item.dX = st->item.dY = nullptr;
    return s;
  }
  *dX = st->item.dX;
  *dY = st->item.dY;
  st->item.dX = st->item.dY = nullptr;
  return FTN_OK;
}

void free_compress_state(CompressState* st) {
  if (!st) return;
  if (st->buf) dev_free(st->ctx, st->buf);
  delete st;
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

extern "C" ftn_status ftn_compress_grad(ftn_ctx ctx, ftn_tensor X, ftn_tensor Y, int n, const int* axes_x,
                                        const int* axes_y, int chi, int arrows, ftn_tensor dXn, ftn_tensor dYn,
                                        ftn_tensor* dX, ftn_tensor* dY) {
  if (!ctx || !X || !Y || !dXn || !dYn || !dX || !dY || (n > 0 && (!axes_x || !axes_y)))
    return set_error(FTN_EINVAL, "null argument");
  if (n < 1) return set_error(FTN_EINVAL, "a bond needs at least one leg pair");
  if (n > MAXR) return set_error(FTN_EINVAL, "too many bond legs");
  std::vector<CompressItem> items(1);
  CompressItem& it = items[0];
  it.X = X;
  it.Y = Y;
  it.n = n;
  for (int i = 0; i < n; ++i) it.ax[i] = axes_x[i], it.ay[i] = axes_y[i];
  it.chi = chi;
  it.arrows = arrows;
  it.gXn = dXn;
  it.gYn = dYn;
  const ftn_status st = compress_batch(ctx, items);
  if (st != FTN_OK) {
    ftn_tensor_free(it.dX);
    ftn_tensor_free(it.dY);
    return st;
  }
  *dX = it.dX;
  *dY = it.dY;
  return FTN_OK;
}

extern "C" ftn_status ftn_compress(ftn_ctx ctx, ftn_tensor* X, ftn_tensor* Y, int n, const int* axes_x,
                                   const int* axes_y, int chi, int arrows, ftn_compress_info* info) {
  return compress_impl(ctx, X, Y, n, axes_x, axes_y, chi, arrows, info);
}
