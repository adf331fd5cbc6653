/*
 * ftn.h -- C ABI of libftn, Z2-graded (fermionic) block-sparse tensor
 * contraction on one NVIDIA GB300 (sm_103a).
 *
 * Method: Gao, Zhai, Gray, Peng, Park, Liu, Kjonstad, Chan, "Fermionic tensor
 * network contraction for arbitrary geometries", arXiv:2410.02215.
 *
 * Conventions used by every entry point
 * -------------------------------------
 * Leg: sector dimensions (d_even, d_odd) and a dual flag.  dual = 1 marks an
 *   incoming ('-') leg, dual = 0 an outgoing ('+') leg (Sec. II.A, symmetry
 *   rule with H = 2).  A bond's arrow runs from its '+' leg to its '-' leg.
 *   Dense index i of a leg has parity [i >= d_even] (even states first).
 * Tensor: rank r <= FTN_MAX_RANK, total parity p in {0, 1} (Sec. II.B).
 *   Its data is one contiguous device buffer of 2^(r-1) blocks (one block of
 *   one element for r = 0 and p = 0; none for r = 0 and p = 1).  Block b has
 *   the parity bitmask m (bit k = sector of leg k) with popcount(m) = p mod 2
 *   and b = m >> 1; blocks are stored in increasing b, each block dense and
 *   row-major in leg order (last leg fastest).  Zero-size blocks take no
 *   space.  Element type is FP64 or FP32.
 * Pairwise contraction op(X, Y) over leg pairs (ax[i], ay[i]): X's contracted
 *   legs are moved to its end in the order ax, Y's to its front in mirror
 *   order, each move a fermionic transposition with sign (-1)^{p_i p_j} per
 *   swapped pair (Eqs. transposition, standardcontract); a pair whose X leg
 *   is outgoing ('+') is contracted against its arrow and carries the bond
 *   parity (-1)^p (locally ordered formalism, Eq. fermionictn2 and the text
 *   after it).  Result legs: X's free legs in order, then Y's.  Contracted
 *   legs must have equal (d_even, d_odd) and opposite duals.
 * Streams: every call is asynchronous on the context's CUDA stream unless
 *   stated otherwise.  The sign-permute and tensor-core GEMM kernels are
 *   launched with programmatic stream serialisation: they may begin while the
 *   kernel before them in the stream is still running, but read or write no
 *   tensor data until it has completed, so stream order is kept for any
 *   earlier work.  Errors are returned as ftn_status; no exception crosses
 *   the ABI; ftn_last_error() gives a message for the calling thread.
 * Ownership: the caller owns the tensors it creates or wraps and releases
 *   them with ftn_tensor_free.  Library-allocated buffers come from the
 *   context's allocator callbacks (or cudaMallocAsync on the context stream
 *   when none are given).
 */
#ifndef FTN_H
#define FTN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FTN_MAX_RANK 16

#if defined(__GNUC__)
#define FTN_API __attribute__((visibility("default")))
#else
#define FTN_API
#endif

typedef struct ftn_ctx_s* ftn_ctx;
typedef struct ftn_tensor_s* ftn_tensor;

typedef enum {
  FTN_OK = 0,
  FTN_EINVAL = -1,       /* bad argument (null pointer, rank, axes, perm)      */
  FTN_ESHAPE = -2,       /* contracted legs differ in (d_even, d_odd)           */
  FTN_EPARITY = -3,      /* parity out of {0,1} or inconsistent                 */
  FTN_EDUAL = -4,        /* contracted legs with equal duals                    */
  FTN_ENOMEM = -5,       /* allocator returned NULL                             */
  FTN_ECUDA = -6,        /* CUDA runtime error                                  */
  FTN_ETIMEOUT = -7,     /* a device-side bounded wait gave up                  */
  FTN_EUNSUPPORTED = -8  /* dtype/precision combination not provided           */
} ftn_status;

typedef enum { FTN_F64 = 0, FTN_F32 = 1 } ftn_dtype;

/* Arithmetic of the sector GEMMs.  FTN_PREC_F64 needs FP64 tensors (DFMA).
 * The others need FP32 tensors and run on the tcgen05 tensor cores with FP32
 * accumulation: TF32 and BF16 round each operand once; TF32X3, BF16X3 and
 * F16X3 split each operand x = hi + lo and sum hi*hi + hi*lo + lo*hi.  F16X3
 * (FP16 hi and lo: 11 + 11 significant bits at the 16-bit tensor rate) keeps
 * TF32X3's accuracy, about 2^-22 of the largest operand entry, while that
 * entry lies between 2^-3 and 2^15 in magnitude (FP16 overflows above
 * 65504, and lo parts below 2^-14 lose bits to the subnormal spacing 2^-24);
 * tensors of the contraction-tree executor are scaled to max |x| = 1. */
typedef enum {
  FTN_PREC_F64 = 0,
  FTN_PREC_TF32 = 1,
  FTN_PREC_BF16 = 2,
  FTN_PREC_TF32X3 = 3,
  FTN_PREC_BF16X3 = 4,
  FTN_PREC_F16X3 = 5
} ftn_prec;

typedef void* (*ftn_alloc_fn)(size_t bytes, void* user);
typedef void (*ftn_free_fn)(void* ptr, void* user);

/* ---- context ----------------------------------------------------------- */

/* Create a context bound to the current CUDA device and to `cuda_stream`
 * (a cudaStream_t, NULL = legacy default stream).  `alloc`/`free` (both or
 * neither) supply device memory for library-owned buffers; `user` is passed
 * back to them.  Returns FTN_ECUDA if no device is usable. */
FTN_API ftn_status ftn_ctx_create(void* cuda_stream, ftn_alloc_fn alloc, ftn_free_fn free_fn, void* user,
                          ftn_ctx* out);
FTN_API ftn_status ftn_ctx_destroy(ftn_ctx ctx);
/* Change the stream later calls are issued on. */
FTN_API ftn_status ftn_ctx_set_stream(ftn_ctx ctx, void* cuda_stream);
/* Tile-width tuning of tensor-core contractions (on when a context is
 * created; no counterpart in the paper, a property of this implementation).
 * While on, the first ftn_tensordot of a contraction with at least 2^30
 * sector flops (not issued under stream capture) also plans its GEMM with the
 * tile width capped at half and a quarter of the default, runs every
 * candidate twice (once timed with CUDA events, synchronising the context
 * stream) and keeps the fastest in the context's plan cache.  The width does
 * not change any result bit.  Off: every plan keeps the default width.
 * Affects plans built after the call.  FTN_EINVAL for a null context. */
FTN_API ftn_status ftn_ctx_set_tuning(ftn_ctx ctx, int on);
/* Synchronise the context stream and report a device-side error recorded
 * since the last call (FTN_ETIMEOUT after a bounded wait gave up). */
FTN_API ftn_status ftn_ctx_synchronize(ftn_ctx ctx);
/* Self-test of device-side failure reporting (no counterpart in the paper;
 * a property of this implementation).  Every wait of the tensor-core GEMM
 * and the staged sign-permute on an mbarrier gives up after 2 s, records a
 * timeout in the context's device error word, lets the other waits of the
 * launch bail out, and the kernel returns instead of hanging; the next
 * ftn_ctx_synchronize reports FTN_ETIMEOUT and clears the word.  This call
 * launches one single-thread kernel on the context stream that waits,
 * through the same bounded-wait code, on an mbarrier phase nothing ever
 * completes, with the limit limit_ns (1e3 to 1e10 ns, else FTN_EINVAL)
 * instead of 2 s.  It faults nothing: the kernel returns after the limit.
 * Results of other work issued on the context between this call and the
 * next ftn_ctx_synchronize are unspecified (their waits may bail out). */
FTN_API ftn_status ftn_ctx_wait_selftest(ftn_ctx ctx, uint64_t limit_ns);
/* Number of kernels this context has launched so far. */
FTN_API int64_t ftn_ctx_launch_count(ftn_ctx ctx);
/* Per-launch timing: while enabled, every kernel launch is bracketed by CUDA
 * events on the context stream and tagged with a label and the algorithmic
 * bytes and flops of that launch (the minimal traffic and the sector-GEMM
 * flops the plan implies).  Enabling clears earlier records. */
FTN_API ftn_status ftn_ctx_profile(ftn_ctx ctx, int enable);
/* Prefix for the labels of later records ("" for none). */
FTN_API ftn_status ftn_ctx_profile_tag(ftn_ctx ctx, const char* tag);
/* Aggregate of the records with label index `idx` (0-based; FTN_EINVAL past
 * the last): label, launch count, summed milliseconds, bytes and flops.
 * Synchronises the context stream. */
FTN_API ftn_status ftn_ctx_profile_read(ftn_ctx ctx, int idx, const char** label, int64_t* launches, double* ms,
                                        double* bytes, double* flops);
/* Message of the last failing call on this thread (never NULL). */
FTN_API const char* ftn_last_error(void);

/* ---- tensors (sector table + device buffer), Sec. II.A-II.B --------------- */

/* Library-allocated tensor, contents undefined.  d_even/d_odd/dual have
 * `rank` entries (ignored for rank 0); parity is 0 or 1. */
FTN_API ftn_status ftn_tensor_create(ftn_ctx ctx, int rank, const int32_t* d_even, const int32_t* d_odd,
                             const uint8_t* dual, int parity, ftn_dtype dtype, ftn_tensor* out);
/* Same metadata over a caller-owned device buffer `dev_data` (borrowed: the
 * caller keeps it alive and frees it; it must hold ftn_tensor_numel
 * elements and be aligned to the element size). */
FTN_API ftn_status ftn_tensor_wrap(ftn_ctx ctx, int rank, const int32_t* d_even, const int32_t* d_odd,
                           const uint8_t* dual, int parity, ftn_dtype dtype, void* dev_data,
                           ftn_tensor* out);
FTN_API ftn_status ftn_tensor_free(ftn_tensor t);
/* Metadata: any output pointer may be NULL; arrays need `rank` entries. */
FTN_API ftn_status ftn_tensor_info(ftn_tensor t, int* rank, int32_t* d_even, int32_t* d_odd, uint8_t* dual,
                           int* parity, ftn_dtype* dtype, int64_t* numel, void** dev_data);
/* Element offsets and parity bitmasks of the 2^(rank-1) blocks in storage
 * order (arrays sized by ftn_tensor_info's rank; *nblocks receives the count). */
FTN_API ftn_status ftn_tensor_block_offsets(ftn_tensor t, int64_t* offsets, uint32_t* masks, int* nblocks);
/* Copy numel elements between a host buffer (pinned or pageable) and the
 * tensor, asynchronously on the context stream. */
FTN_API ftn_status ftn_tensor_upload(ftn_ctx ctx, ftn_tensor t, const void* host);
FTN_API ftn_status ftn_tensor_download(ftn_ctx ctx, ftn_tensor t, void* host);

/* ---- sign-permute (Eq. transposition) ------------------------------------ */

/* Fermionic transposition: out leg u = in leg perm[u]; every block is moved
 * and multiplied by (-1)^{sum of p_a p_b over leg pairs whose order the
 * permutation inverts}.  *out is created (same dtype) unless it is non-NULL
 * on entry, in which case it must already have the permuted metadata and
 * 16-byte aligned data (else FTN_EINVAL). */
FTN_API ftn_status ftn_tensor_transpose(ftn_ctx ctx, ftn_tensor t, const int* perm, ftn_tensor* out);
/* Hermitian conjugate of one tensor (Sec. II.C): leg order reversed, duals
 * flipped, no sign (real data). */
FTN_API ftn_status ftn_tensor_dagger(ftn_ctx ctx, ftn_tensor t, ftn_tensor* out);

/* ---- fermionic tensordot (Eqs. standardcontract, fermiswap, Sec. IV.A) --- */

/* C = op(A, B) over n leg pairs (axes_a[i], axes_b[i]), with the bond parity
 * (-1)^p applied additionally on every leg k of A with bit k of flip_a set
 * and every leg k of B with bit k of flip_b set (the g tensors a global-order
 * move accumulates, Sec. II.C).  If out_perm is not NULL the result is
 * fermionically transposed to out leg u = result leg out_perm[u].  A and B
 * must have the same dtype; prec selects the GEMM arithmetic.  *C is created
 * unless non-NULL on entry (then it must match the result's metadata and its
 * data must be 16-byte aligned, else FTN_EINVAL).
 * n = 0 gives the outer product. */
FTN_API ftn_status ftn_tensordot(ftn_ctx ctx, ftn_tensor A, ftn_tensor B, int n, const int* axes_a,
                         const int* axes_b, uint64_t flip_a, uint64_t flip_b, const int* out_perm,
                         ftn_prec prec, ftn_tensor* C);

/* ---- adjoint of the tensordot (the contraction is linear in each operand) - */

/* Gradients of L = sum(G * C) with C = ftn_tensordot(A, B, n, axes_a, axes_b,
 * flip_a, flip_b, out_perm): G holds dL/dC and must have exactly C's metadata
 * (legs after out_perm, parity p_A + p_B) and A's dtype.  dA (if dA is not
 * NULL) gets A's metadata and dL/dA, dB (if not NULL) B's and dL/dB; each is
 * created unless non-NULL on entry (then its metadata must match and its
 * data be 16-byte aligned).  Every
 * block pair of the forward product carries one sign (transposition of the
 * operands into the contraction order with the arrow and extra bond
 * parities, and of the result into out_perm); the adjoint applies the same
 * signs, so <dA, A> = <G, C> = <dB, B>.  prec: as for ftn_tensordot.
 * Gradients of contractions serve the variational optimisation of fermionic
 * PEPS that the paper refers to (Sec. II.D); the paper prints no adjoint, and
 * this is a hand-written one.  Errors: as ftn_tensordot, and FTN_ESHAPE when
 * G's legs or parity differ from C's. */
FTN_API ftn_status ftn_tensordot_grad(ftn_ctx ctx, ftn_tensor A, ftn_tensor B, ftn_tensor G, int n,
                                      const int* axes_a, const int* axes_b, uint64_t flip_a, uint64_t flip_b,
                                      const int* out_perm, ftn_prec prec, ftn_tensor* dA, ftn_tensor* dB);

/* ---- tensordot without device allocation ---------------------------------- */

/* The paper has no counterpart of this entry point; it exists for callers
 * that cannot allocate device memory, directly or through the library:
 * plug-in hosts that hand a library only the buffers they reserved up front,
 * and processes whose device memory belongs to another framework's allocator
 * that must not be grown behind its back.
 *
 * Same operation as ftn_tensordot (without the extra bond-parity masks) on
 * raw device buffers: A and B are described by their legs and parity and
 * hold their blocks in the layout above (element type `dtype`); the result
 * (legs: free legs of A then of B, permuted by out_perm when not NULL) is
 * written to the caller-owned device buffer `c` of at least c_capacity
 * elements.  Every temporary (fused sector matrices, plan tables, error
 * word) lives in one file-scope static device array of
 * FTN_NOALLOC_SCRATCH_BYTES that every GPU loading the library keeps until
 * the process exits; the call never calls cudaMalloc, cudaFree or any other
 * device-allocating routine (host bookkeeping uses the C++ heap).  A
 * contraction that needs more scratch than the array holds, or a result
 * larger than c_capacity, is rejected with FTN_EINVAL and a message.  The
 * first call on each device (that device current)
 * looks up the array's device address once.  All calls share the array and
 * it keeps the last call's contents.  Work of two calls overlapping on the
 * GPU would race on it; the call prevents that by serialising callers with a
 * host lock and by returning only after its work on `cuda_stream` (and
 * everything queued there before it) has finished: it copies its plan tables
 * from pageable host memory on the stream and synchronises the stream at the
 * end to read the device error word (FTN_ETIMEOUT when a bounded wait of the
 * kernels gave up).  Tile-width tuning is off on this path. */
#define FTN_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
FTN_API ftn_status ftn_tensordot_noalloc(void* cuda_stream, int rank_a, const int32_t* d_even_a,
                                         const int32_t* d_odd_a, const uint8_t* dual_a, int parity_a,
                                         const void* a, int rank_b, const int32_t* d_even_b,
                                         const int32_t* d_odd_b, const uint8_t* dual_b, int parity_b,
                                         const void* b, ftn_dtype dtype, int n, const int* axes_a,
                                         const int* axes_b, const int* out_perm, ftn_prec prec, void* c,
                                         int64_t c_capacity);

/* ---- bond compression (Sec. II.A symmetric QR/SVD, Sec. III) ------------- */

typedef struct {
  int kept[2];          /* new bond (d_even, d_odd)                           */
  int rank[2];          /* numerical rank of each bond-parity sector          */
  double discarded_sq;  /* sum of the squared discarded singular values       */
  double total_sq;      /* sum of all squared singular values                 */
  double s_max;         /* largest singular value                             */
  double s_cut;         /* smallest kept singular value (0 if none kept)      */
  double s_next;        /* largest discarded singular value (0 if none)       */
  int jacobi_sweeps;    /* sweeps the one-sided Jacobi SVD needed (diagnostic) */
} ftn_compress_info;

/* Compress the bond formed by legs axes_x of *X paired with axes_y of *Y to at
 * most chi states: per bond-parity sector the R factors of X = [free | bond]
 * and of Y^T = [free | bond]^T, the core M = R_X R_Y^T, its SVD, the chi
 * largest singular values pooled over both sectors (ties to the even sector,
 * then the lower index), and the new pair X' = [free_X | new], Y' = [new |
 * free_Y] with op(X', Y') the truncated op(X, Y) (the new leg is incoming on
 * X' and outgoing on Y').  Singular values below 1e-14 * s_max are numerical
 * zeros and never kept.  `arrows` = 0 contracts the bond without the arrow
 * parity (plain ordered contraction F(XY) of the global formalism).  *X and
 * *Y are replaced by new library-owned tensors and the old ones freed.  FP64
 * arithmetic throughout.  Synchronises twice (the nonzero rows of the R
 * factors and the kept dimensions are data). */
FTN_API ftn_status ftn_compress(ftn_ctx ctx, ftn_tensor* X, ftn_tensor* Y, int n, const int* axes_x,
                        const int* axes_y, int chi, int arrows, ftn_compress_info* info);

/* Adjoint of ftn_compress (the gradient of the Sec. II.A compression, which
 * the paper does not differentiate): for a scalar L of the compressed pair
 * (X', Y') = ftn_compress(X, Y, ...) with the same arguments, given the
 * cotangents dXn = dL/dX' and dYn = dL/dY' (FP64 tensors with the legs and
 * parity of X' and Y'), returns dX = dL/dX and dY = dL/dY as new
 * library-owned tensors with X's and Y's legs.  X and Y are borrowed and left
 * unchanged; the forward compression is recomputed (its kept set and
 * factors).  Per bond-parity sector: the reverse-mode rules of the column
 * scalings, of the thin SVD of the core (F-matrix 1/(s_j^2 - s_i^2) over every
 * singular pair with a kept member, projections onto the complements of the
 * kept vectors) and of the R factors, then the adjoint of the
 * sign-permutes.  Defined where the compression is differentiable: a gap at
 * the truncation cut, distinct nonzero singular values, full-rank sector
 * blocks; a block whose factor drops rows gives FTN_EUNSUPPORTED, cotangents
 * of the wrong shape FTN_ESHAPE.  Singular values of a core at or below
 * 1e-12 of its largest count as zero: their directions are left to the
 * complements the rule projects onto (a relative error of that order).  A
 * loss that depends on the gauge of the new bond (signs of its states) has
 * no well-defined gradient.  FP64 throughout; synchronises as ftn_compress. */
FTN_API ftn_status ftn_compress_grad(ftn_ctx ctx, ftn_tensor X, ftn_tensor Y, int n, const int* axes_x,
                             const int* axes_y, int chi, int arrows, ftn_tensor dXn, ftn_tensor dYn,
                             ftn_tensor* dX, ftn_tensor* dY);

/* ---- contraction tree executor (Fig. 1, Secs. II.C-II.D, III) ------------ */

typedef enum { FTN_POLICY_EXACT = 0, FTN_POLICY_EARLY = 1, FTN_POLICY_LATE = 2 } ftn_policy;

typedef struct {
  int n_tensors;
  const ftn_tensor* tensors; /* borrowed, left untouched                       */
  int n_bonds;
  const int32_t* bonds;      /* 4 per bond: tensor1, leg1, tensor2, leg2        */
  const int32_t* positions;  /* NULL: locally ordered; else global positions    */
} ftn_network;

typedef struct {
  int n_steps;               /* n_tensors - 1                                  */
  const int32_t* pairs;      /* 2 per step, SSA ids: inputs 0..n-1, step s -> n+s */
  ftn_policy policy;
  int chi;                   /* bond cap for EARLY/LATE                        */
} ftn_tree;

/* Contract a closed network along the tree.  Locally ordered when
 * positions == NULL (bond parity when a bond is contracted against its
 * arrow; each odd tensor carries a size-1 odd dummy leg (Sec. II.D), and
 * the dummy legs left at the end are sorted by decreasing tensor index,
 * which gives the value of the globally ordered network with the tensors
 * in index order); globally ordered otherwise (the later tensor is moved past the
 * tensors between, each shared bond passed carrying g and each odd tensor
 * passed a phase, then plain F).  Late policy compresses, just before a
 * step, every other bond of both operands whose dimension exceeds chi;
 * early policy compresses the new tensor's bonds right after the step;
 * neighbours in increasing id.  After every step the new tensor is divided
 * by its largest |entry| and the natural log accumulated: value =
 * (*mantissa) * exp(*log_scale).  Synchronises at the end. */
FTN_API ftn_status ftn_contract(ftn_ctx ctx, const ftn_network* net, const ftn_tree* tree, ftn_prec prec,
                        double* mantissa, double* log_scale);

/* Contract `count` independent closed networks (for instance the cluster
 * networks of all energy terms of many states, Sec. V): nets[i] along
 * trees[i], each exactly as ftn_contract would, with results
 * mantissa[i] * exp(log_scale[i]) (host arrays of count doubles).  The
 * networks advance in lock step -- round s runs step s of every network that
 * has one -- and every stage of a round (sign-permutes, grouped sector GEMMs,
 * the compressions before or after the step, normalisation) is one launch per
 * kernel over all networks, so the launch count grows with the number of
 * steps, not with the number of networks.  Each network keeps the arithmetic
 * it has alone (plans, tiles, reduction orders): results are bit-identical
 * to count separate ftn_contract calls.  All networks share `prec`; trees may
 * differ in policy and chi.  Memory: the live tensors of all networks are
 * held at once.  Errors: as ftn_contract, for the first network that fails
 * validation (nothing is launched then); FTN_EINVAL when count < 0 or an
 * array is NULL with count > 0.  Synchronises at the end and, with
 * compression, twice per sub-round of compressions. */
FTN_API ftn_status ftn_contract_batch(ftn_ctx ctx, int count, const ftn_network* nets, const ftn_tree* trees,
                              ftn_prec prec, double* mantissa, double* log_scale);

/* ftn_contract_batch with the values left on the device and no host
 * synchronisation: d_out (2 * count doubles of device memory, owned by the
 * caller) receives d_out[2 i] = the mantissa of network i (its sign
 * included) and d_out[2 i + 1] = its natural-log scale, written in the order
 * of ctx's stream.  The call may be captured into a CUDA graph on ctx's
 * stream (stream capture) -- all local terms of many networks replayed as one
 * graph launch -- provided every contraction's plan already exists on this
 * context (each network contracted once before, same shapes) and no
 * compression runs (a compression reads its kept dimensions back to the
 * host); otherwise FTN_EUNSUPPORTED, and the capture holds a partial graph
 * that must not be replayed.  Tables uploaded during a capture come from
 * pinned host copies that the context keeps until it is destroyed; a graph
 * reads the networks' tensors at replay, so it stays valid while they and
 * the context live (their values may change between replays).  Errors
 * otherwise as ftn_contract_batch. */
FTN_API ftn_status ftn_contract_batch_async(ftn_ctx ctx, int count, const ftn_network* nets, const ftn_tree* trees,
                                    ftn_prec prec, double* d_out);

/* Value of a closed network of even FP64 tensors and its gradient with
 * respect to every tensor of the network (each tensor an independent input,
 * a bra that is the dagger of a ket included): *value = v (plain FP64, no
 * per-step normalisation, so v must stay within FP64's range) and grads[i] =
 * dv/dT_i, a new library-owned tensor with T_i's legs, for i < n_tensors.
 * The forward is ftn_contract's walk of the tree (same pairs, flips, phases,
 * and late / early compressions of the same bonds); the backward passes each
 * result's cotangent to its operands by ftn_tensordot_grad and each
 * compression's by ftn_compress_grad, in reverse order (the paper gives no
 * gradient; variational fPEPS optimisation needs one, Sec. II.D).  Defined
 * where every compression is differentiable (ftn_compress_grad's
 * conditions; FTN_EUNSUPPORTED otherwise) and for even tensors only.
 * checkpoint = 0 keeps every intermediate until the call returns.
 * checkpoint = k > 0 keeps only the walk's state every k steps (its live
 * tensors and the executor's leg bookkeeping) and frees the rest; the
 * backward replays each segment of k steps from its checkpoint, keeping that
 * segment's operands, before passing the cotangents through it -- one extra
 * forward pass (all but the last segment) for memory of the checkpoints and
 * one segment.  The replay is bit-identical to the first walk (the kernels
 * are deterministic), so the value and gradient do not depend on k.
 * FTN_EINVAL for k < 0.  Synchronises at the end and as every compression
 * does. */
FTN_API ftn_status ftn_contract_grad(ftn_ctx ctx, const ftn_network* net, const ftn_tree* tree, int checkpoint,
                             double* value, ftn_tensor* grads);

/* ---- expectation values of local terms (Sec. V) --------------------------- */

/* Per-term ratios and their sums from contracted network values.  Network i
 * has the value mantissa[i] * exp(log_scale[i]) (as ftn_contract returns
 * it); term t is the ratio ratios[t] = value(num[t]) / value(den[t]) =
 * (mantissa[num[t]] / mantissa[den[t]]) * exp(log_scale[num[t]] -
 * log_scale[den[t]]) -- <Psi|h_t|Psi> / <Psi|Psi> when num[t] is the term's
 * network and den[t] the norm network (Sec. V; every term of a whole-state
 * energy shares one norm network, a cluster term of Fig. 4b has its own).
 * The terms are split into n_groups consecutive groups (group g ends before
 * term group_end[g]; non-decreasing, at most n_terms) and energies[g]
 * receives the FP64 sum of its ratios, added in term order (one group per
 * state; terms after the last group_end belong to none).  ratios may be
 * NULL.  Host arithmetic only: no device is touched, the result depends on
 * nothing but the inputs.  FTN_EINVAL for an index out of [0, count), a
 * null array that is needed, or a denominator whose value is zero or not
 * finite. */
FTN_API ftn_status ftn_energy_reduce(int count, const double* mantissa, const double* log_scale, int n_terms,
                                     const int32_t* num, const int32_t* den, int n_groups, const int32_t* group_end,
                                     double* ratios, double* energies);

/* Contract the `count` closed networks nets[i] along trees[i] and reduce
 * them as ftn_energy_reduce does.  The n_ctx contexts (same device, each on
 * its own stream; ctxs[0] owns or may have produced the input tensors) each
 * run on one host thread and take the next network -- or, with batch > 0,
 * the next run of up to `batch` consecutive networks, contracted in lock
 * step by ftn_contract_batch -- from a shared counter; the first context's
 * stream is synchronised before any other reads the inputs.  Every network
 * is contracted exactly as ftn_contract contracts it, whatever context or
 * batch it lands in, so the values and sums are the same for any n_ctx and
 * batch.  mantissa / log_scale (count entries, may be NULL) receive the
 * network values.  Errors: those of ftn_contract / ftn_contract_batch (the
 * first one met; the other threads stop taking work) and of
 * ftn_energy_reduce.  Returns after every network has been contracted. */
FTN_API ftn_status ftn_energy(int n_ctx, const ftn_ctx* ctxs, int count, const ftn_network* nets,
                              const ftn_tree* trees, ftn_prec prec, int batch, double* mantissa, double* log_scale,
                              int n_terms, const int32_t* num, const int32_t* den, int n_groups,
                              const int32_t* group_end, double* ratios, double* energies);

/* ---- Hubbard terms (Eq. fermi-hubbard-ham) -------------------------------- */

/* Even operator tensors for <Psi| h_t |Psi> (physical leg (2,2): 0 = |0>,
 * 1 = |up dn>, 2 = |up>, 3 = |dn>).  kind 0: hopping -t sum_s (c+_is c_js +
 * h.c.) on a bond i < j, legs [i', j', j, i] with duals (0, 0, 1, 1); entries
 * are matrix elements in the ordered creation-string basis with site i
 * first.  kind 1: on-site U n_up n_dn, legs [i', i], duals (0, 1). */
FTN_API ftn_status ftn_hubbard_term(ftn_ctx ctx, int kind, double t, double u, ftn_dtype dtype,
                            ftn_tensor* out);

#ifdef __cplusplus
}
#endif
#endif /* FTN_H */
