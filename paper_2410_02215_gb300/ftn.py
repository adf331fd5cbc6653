"""Thin ctypes binding of libftn (include/ftn.h).

Argument marshalling only: every step of a contraction, transposition or
compression runs in libftn's CUDA kernels.  PyTorch supplies device memory
(through the context's allocator callbacks) and the CUDA stream.  Importing
this module fails loudly when the compiled library is missing.
"""
from __future__ import annotations

import ctypes as C
import itertools
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libftn.so")

FTN_MAX_RANK = 16
F64, F32 = 0, 1
PREC_F64, PREC_TF32, PREC_BF16, PREC_TF32X3, PREC_BF16X3, PREC_F16X3 = 0, 1, 2, 3, 4, 5
PREC_NAMES = {"f64": PREC_F64, "tf32": PREC_TF32, "bf16": PREC_BF16, "tf32x3": PREC_TF32X3, "bf16x3": PREC_BF16X3,
              "f16x3": PREC_F16X3}
POLICY_EXACT, POLICY_EARLY, POLICY_LATE = 0, 1, 2
POLICY_NAMES = {"exact": POLICY_EXACT, "early": POLICY_EARLY, "late": POLICY_LATE}
STATUS = {0: "FTN_OK", -1: "FTN_EINVAL", -2: "FTN_ESHAPE", -3: "FTN_EPARITY", -4: "FTN_EDUAL", -5: "FTN_ENOMEM",
          -6: "FTN_ECUDA", -7: "FTN_ETIMEOUT", -8: "FTN_EUNSUPPORTED"}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class FtnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class CompressInfo(C.Structure):
    _fields_ = [("kept", C.c_int * 2), ("rank", C.c_int * 2), ("discarded_sq", C.c_double),
                ("total_sq", C.c_double), ("s_max", C.c_double), ("s_cut", C.c_double), ("s_next", C.c_double),
                ("jacobi_sweeps", C.c_int)]


class Network(C.Structure):
    _fields_ = [("n_tensors", C.c_int), ("tensors", C.POINTER(C.c_void_p)), ("n_bonds", C.c_int),
                ("bonds", C.POINTER(C.c_int32)), ("positions", C.POINTER(C.c_int32))]


class Tree(C.Structure):
    _fields_ = [("n_steps", C.c_int), ("pairs", C.POINTER(C.c_int32)), ("policy", C.c_int), ("chi", C.c_int)]


_lib = None


def lib():
    """The loaded libftn (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libftn is not built ({LIB_PATH} missing); run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    vp, i32p, u8p, i64p, u32p = C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_uint8), C.POINTER(C.c_int64), C.POINTER(C.c_uint32)
    ip = C.POINTER(C.c_int)
    sigs = {
        "ftn_ctx_create": [vp, ALLOC_FN, FREE_FN, vp, C.POINTER(vp)],
        "ftn_ctx_destroy": [vp],
        "ftn_ctx_set_stream": [vp, vp],
        "ftn_ctx_set_tuning": [vp, C.c_int],
        "ftn_ctx_synchronize": [vp],
        "ftn_ctx_wait_selftest": [vp, C.c_uint64],
        "ftn_tensor_create": [vp, C.c_int, i32p, i32p, u8p, C.c_int, C.c_int, C.POINTER(vp)],
        "ftn_tensor_wrap": [vp, C.c_int, i32p, i32p, u8p, C.c_int, C.c_int, vp, C.POINTER(vp)],
        "ftn_tensor_free": [vp],
        "ftn_tensor_info": [vp, ip, i32p, i32p, u8p, ip, ip, i64p, C.POINTER(vp)],
        "ftn_tensor_block_offsets": [vp, i64p, u32p, ip],
        "ftn_tensor_upload": [vp, vp, vp],
        "ftn_tensor_download": [vp, vp, vp],
        "ftn_tensor_transpose": [vp, vp, ip, C.POINTER(vp)],
        "ftn_tensor_dagger": [vp, vp, C.POINTER(vp)],
        "ftn_tensordot": [vp, vp, vp, C.c_int, ip, ip, C.c_uint64, C.c_uint64, ip, C.c_int, C.POINTER(vp)],
        "ftn_tensordot_grad": [vp, vp, vp, vp, C.c_int, ip, ip, C.c_uint64, C.c_uint64, ip, C.c_int, C.POINTER(vp),
                               C.POINTER(vp)],
        "ftn_compress": [vp, C.POINTER(vp), C.POINTER(vp), C.c_int, ip, ip, C.c_int, C.c_int, C.POINTER(CompressInfo)],
        "ftn_compress_grad": [vp, vp, vp, C.c_int, ip, ip, C.c_int, C.c_int, vp, vp, C.POINTER(vp), C.POINTER(vp)],
        "ftn_contract": [vp, C.POINTER(Network), C.POINTER(Tree), C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)],
        "ftn_contract_batch": [vp, C.c_int, C.POINTER(Network), C.POINTER(Tree), C.c_int, C.POINTER(C.c_double),
                               C.POINTER(C.c_double)],
        "ftn_contract_batch_async": [vp, C.c_int, C.POINTER(Network), C.POINTER(Tree), C.c_int, vp],
        "ftn_contract_grad": [vp, C.POINTER(Network), C.POINTER(Tree), C.c_int, C.POINTER(C.c_double), C.POINTER(vp)],
        "ftn_hubbard_term": [vp, C.c_int, C.c_double, C.c_double, C.c_int, C.POINTER(vp)],
        "ftn_energy_reduce": [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int, i32p, i32p, C.c_int,
                              i32p, C.POINTER(C.c_double), C.POINTER(C.c_double)],
        "ftn_energy": [C.c_int, C.POINTER(vp), C.c_int, C.POINTER(Network), C.POINTER(Tree), C.c_int, C.c_int,
                       C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int, i32p, i32p, C.c_int, i32p,
                       C.POINTER(C.c_double), C.POINTER(C.c_double)],
    }
    for name, args in sigs.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.ftn_last_error.argtypes = []
    L.ftn_last_error.restype = C.c_char_p
    L.ftn_ctx_launch_count.argtypes = [vp]
    L.ftn_ctx_launch_count.restype = C.c_int64
    L.ftn_ctx_profile.argtypes = [vp, C.c_int]
    L.ftn_ctx_profile.restype = C.c_int
    L.ftn_ctx_profile_tag.argtypes = [vp, C.c_char_p]
    L.ftn_ctx_profile_tag.restype = C.c_int
    L.ftn_ctx_profile_read.argtypes = [vp, C.c_int, C.POINTER(C.c_char_p), C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                       C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.ftn_ctx_profile_read.restype = C.c_int
    _lib = L
    return L


def _check(st):
    if st != 0:
        raise FtnError(st, lib().ftn_last_error().decode())


def _i32(seq):
    seq = list(seq)
    return (C.c_int32 * max(1, len(seq)))(*seq)


def _int(seq):
    seq = list(seq)
    return (C.c_int * max(1, len(seq)))(*seq)


class Context:
    """ftn_ctx bound to a torch CUDA stream.  Library-owned device memory comes
    from the device's stream-ordered pool (cudaMallocAsync, native, no Python
    on the allocation path) or, with use_torch_allocator=True, from torch's
    caching allocator through the context's allocator callbacks."""

    def __init__(self, stream=None, use_torch_allocator=False):
        import torch

        self._torch = torch
        self.device = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._keep = []
        if use_torch_allocator:
            dev, st = self.device, self.stream

            def _alloc(nbytes, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, st)
                except Exception:  # allocation failure becomes FTN_ENOMEM
                    return None

            def _free(ptr, user):
                if ptr:
                    try:
                        torch.cuda.caching_allocator_delete(ptr)
                    except Exception:  # interpreter shutdown: torch already finalised
                        pass

            a, f = ALLOC_FN(_alloc), FREE_FN(_free)
            self._keep += [a, f]
        else:
            a, f = ALLOC_FN(0), FREE_FN(0)
        h = C.c_void_p()
        _check(lib().ftn_ctx_create(C.c_void_p(self.stream.cuda_stream), a, f, None, C.byref(h)))
        self.handle = h
        self._tensors = weakref.WeakSet()  # tensors to release before the context goes

    def synchronize(self):
        _check(lib().ftn_ctx_synchronize(self.handle))

    def set_stream(self, stream):
        """Launch on another torch CUDA stream from now on (ftn_ctx_set_stream),
        e.g. a stream under CUDA-graph capture."""
        _check(lib().ftn_ctx_set_stream(self.handle, C.c_void_p(stream.cuda_stream)))
        self.stream = stream

    def set_tuning(self, on):
        """Tile-width tuning of large tensor-core contractions on their first
        use (ftn_ctx_set_tuning; on by default)."""
        _check(lib().ftn_ctx_set_tuning(self.handle, 1 if on else 0))

    def wait_selftest(self, limit_ns):
        """Launch the bounded-wait self-test kernel (ftn_ctx_wait_selftest)."""
        _check(lib().ftn_ctx_wait_selftest(self.handle, int(limit_ns)))

    def launches(self):
        return int(lib().ftn_ctx_launch_count(self.handle))

    def profile(self, enable=True):
        _check(lib().ftn_ctx_profile(self.handle, 1 if enable else 0))

    def profile_tag(self, tag):
        _check(lib().ftn_ctx_profile_tag(self.handle, tag.encode()))

    def profile_read(self):
        """[{label, launches, ms, bytes, flops}] aggregated per label."""
        out = []
        i = 0
        while True:
            lab, n = C.c_char_p(), C.c_int64()
            ms, by, fl = C.c_double(), C.c_double(), C.c_double()
            st = lib().ftn_ctx_profile_read(self.handle, i, C.byref(lab), C.byref(n), C.byref(ms), C.byref(by), C.byref(fl))
            if st != 0:
                break
            out.append({"label": lab.value.decode(), "launches": n.value, "ms": ms.value, "bytes": by.value,
                        "flops": fl.value})
            i += 1
        return out

    def close(self):
        if self.handle:
            for t in list(self._tensors):
                t.free()
            lib().ftn_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _CAI:
    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


class Tensor:
    """A graded tensor in libftn's packed sector layout (ftn_tensor)."""

    def __init__(self, ctx, handle, keep=None):
        self.ctx = ctx
        self.handle = handle
        self._keep = keep  # borrowed storage kept alive for wrapped tensors
        ctx._tensors.add(self)
        r = C.c_int()
        d0 = (C.c_int32 * FTN_MAX_RANK)()
        d1 = (C.c_int32 * FTN_MAX_RANK)()
        du = (C.c_uint8 * FTN_MAX_RANK)()
        par, dt, n, ptr = C.c_int(), C.c_int(), C.c_int64(), C.c_void_p()
        _check(lib().ftn_tensor_info(handle, C.byref(r), d0, d1, du, C.byref(par), C.byref(dt), C.byref(n), C.byref(ptr)))
        self.rank = r.value
        self.legs = [(d0[k], d1[k], du[k]) for k in range(self.rank)]
        self.parity = par.value
        self.dtype = dt.value
        self.numel = n.value
        self.ptr = ptr.value or 0

    # ---- construction ----
    @staticmethod
    def _meta(legs):
        r = len(legs)
        return r, _i32([l[0] for l in legs]), _i32([l[1] for l in legs]), (C.c_uint8 * max(1, r))(*[l[2] for l in legs])

    @classmethod
    def empty(cls, ctx, legs, parity, dtype=F64):
        r, d0, d1, du = cls._meta(legs)
        h = C.c_void_p()
        _check(lib().ftn_tensor_create(ctx.handle, r, d0, d1, du, parity, dtype, C.byref(h)))
        return cls(ctx, h)

    @classmethod
    def wrap(cls, ctx, legs, parity, storage, dtype=None):
        """Borrow a contiguous torch CUDA tensor as the data buffer."""
        torch = ctx._torch
        if dtype is None:
            dtype = F64 if storage.dtype == torch.float64 else F32
        r, d0, d1, du = cls._meta(legs)
        h = C.c_void_p()
        _check(lib().ftn_tensor_wrap(ctx.handle, r, d0, d1, du, parity, dtype, C.c_void_p(storage.data_ptr()), C.byref(h)))
        return cls(ctx, h, keep=storage)

    def block_table(self):
        nb = 1 << max(self.rank - 1, 0)
        offs = (C.c_int64 * max(1, nb))()
        masks = (C.c_uint32 * max(1, nb))()
        cnt = C.c_int()
        _check(lib().ftn_tensor_block_offsets(self.handle, offs, masks, C.byref(cnt)))
        return [(int(masks[b]), int(offs[b])) for b in range(cnt.value)]

    def bits_of(self, mask):
        return tuple((mask >> k) & 1 for k in range(self.rank))

    def block_shape(self, bits):
        return tuple(l[1] if b else l[0] for l, b in zip(self.legs, bits))

    def np_dtype(self):
        return np.float64 if self.dtype == F64 else np.float32

    def view(self):
        """Zero-copy torch view of the packed buffer (valid while self lives)."""
        torch = self.ctx._torch
        typestr = "<f8" if self.dtype == F64 else "<f4"
        if self.numel == 0:
            return torch.empty(0, dtype=torch.float64 if self.dtype == F64 else torch.float32, device="cuda")
        return torch.as_tensor(_CAI(self.ptr, self.numel, typestr), device="cuda")

    def upload(self, flat):
        flat = np.ascontiguousarray(flat, dtype=self.np_dtype())
        assert flat.size == self.numel
        _check(lib().ftn_tensor_upload(self.ctx.handle, self.handle, flat.ctypes.data_as(C.c_void_p)))
        self.ctx.synchronize()

    def download(self):
        out = np.empty(self.numel, dtype=self.np_dtype())
        _check(lib().ftn_tensor_download(self.ctx.handle, self.handle, out.ctypes.data_as(C.c_void_p)))
        self.ctx.synchronize()
        return out

    @classmethod
    def from_blocks(cls, ctx, legs, parity, blocks, dtype=F64):
        """Pack ``[(bits, ndarray), ...]`` into a new library tensor."""
        t = cls.empty(ctx, legs, parity, dtype)
        flat = np.zeros(t.numel, dtype=t.np_dtype())
        table = {t.bits_of(m): off for m, off in t.block_table()}
        for bits, arr in blocks:
            arr = np.asarray(arr)
            off = table[tuple(int(b) for b in bits)]
            flat[off:off + arr.size] = arr.reshape(-1)
        t.upload(flat)
        return t

    def to_blocks(self):
        flat = self.download()
        out = []
        for m, off in self.block_table():
            bits = self.bits_of(m)
            shp = self.block_shape(bits)
            n = int(np.prod(shp)) if shp else 1
            out.append((bits, flat[off:off + n].reshape(shp).astype(np.float64)))
        return out

    def free(self):
        if self.handle:
            if self.ctx.handle:  # a closed context has already released its tensors
                lib().ftn_tensor_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ---- operations -------------------------------------------------------------------
def _prec(p):
    return PREC_NAMES[p] if isinstance(p, str) else int(p)


def tensordot(ctx, a, b, axes_a, axes_b, flip_a=0, flip_b=0, out_perm=None, prec="f64", out=None):
    h = C.c_void_p(out.handle.value if out is not None else None)
    n = len(axes_a)
    op = _int(out_perm) if out_perm is not None else None
    _check(lib().ftn_tensordot(ctx.handle, a.handle, b.handle, n, _int(axes_a), _int(axes_b), int(flip_a), int(flip_b),
                               op, _prec(prec), C.byref(h)))
    return out if out is not None else Tensor(ctx, h)


def tensordot_grad(ctx, a, b, g, axes_a, axes_b, flip_a=0, flip_b=0, out_perm=None, prec="f64", wrt=("a", "b"),
                   out_a=None, out_b=None):
    """Gradients (dA, dB) of sum(G * C) for C = tensordot(a, b, ...) with the
    same arguments; g has C's metadata.  Entries of `wrt` not requested come
    back as None; out_a / out_b may be preallocated tensors."""
    n = len(axes_a)
    op = _int(out_perm) if out_perm is not None else None
    ha = C.c_void_p(out_a.handle.value if out_a is not None else None)
    hb = C.c_void_p(out_b.handle.value if out_b is not None else None)
    _check(lib().ftn_tensordot_grad(ctx.handle, a.handle, b.handle, g.handle, n, _int(axes_a), _int(axes_b),
                                    int(flip_a), int(flip_b), op, _prec(prec),
                                    C.byref(ha) if "a" in wrt else None, C.byref(hb) if "b" in wrt else None))
    da = (out_a if out_a is not None else Tensor(ctx, ha)) if "a" in wrt else None
    db = (out_b if out_b is not None else Tensor(ctx, hb)) if "b" in wrt else None
    return da, db


def _numel(legs, parity):
    """Stored elements of a graded tensor: sum over parity-allowed blocks."""
    tot = 0
    for bits in itertools.product((0, 1), repeat=len(legs)):
        if sum(bits) % 2 == parity:
            n = 1
            for (d0, d1, _), bt in zip(legs, bits):
                n *= d1 if bt else d0
            tot += n
    return tot


def _result_legs(legs_a, legs_b, axes_a, axes_b, out_perm):
    free = [l for k, l in enumerate(legs_a) if k not in axes_a] + [l for k, l in enumerate(legs_b) if k not in axes_b]
    return [free[p] for p in out_perm] if out_perm is not None else free


class _TensordotFn:
    """torch.autograd.Function over flat block-data tensors (built lazily so
    that importing this module does not need torch)."""

    _cls = None

    @classmethod
    def get(cls):
        if cls._cls is None:
            import torch

            class Fn(torch.autograd.Function):
                @staticmethod
                def forward(fctx, a_data, b_data, spec):
                    ctx, la, pa, lb, pb, axa, axb, fa, fb, perm, prec = spec
                    dt = F64 if a_data.dtype == torch.float64 else F32
                    a = Tensor.wrap(ctx, la, pa, a_data, dt)
                    b = Tensor.wrap(ctx, lb, pb, b_data, dt)
                    lc = _result_legs(la, lb, axa, axb, perm)
                    c_data = torch.empty(_numel(lc, pa ^ pb), dtype=a_data.dtype, device=a_data.device)
                    c = Tensor.wrap(ctx, lc, pa ^ pb, c_data, dt)
                    tensordot(ctx, a, b, axa, axb, fa, fb, perm, prec, out=c)
                    fctx.save_for_backward(a_data, b_data)
                    fctx.spec = spec
                    return c_data

                @staticmethod
                def backward(fctx, g_data):
                    a_data, b_data = fctx.saved_tensors
                    ctx, la, pa, lb, pb, axa, axb, fa, fb, perm, prec = fctx.spec
                    dt = F64 if a_data.dtype == torch.float64 else F32
                    g_data = g_data.contiguous()
                    a = Tensor.wrap(ctx, la, pa, a_data, dt)
                    b = Tensor.wrap(ctx, lb, pb, b_data, dt)
                    g = Tensor.wrap(ctx, _result_legs(la, lb, axa, axb, perm), pa ^ pb, g_data, dt)
                    wa, wb = fctx.needs_input_grad[0], fctx.needs_input_grad[1]
                    da_data = torch.empty_like(a_data) if wa else None
                    db_data = torch.empty_like(b_data) if wb else None
                    wrt = ("a",) * bool(wa) + ("b",) * bool(wb)
                    if wrt:
                        tensordot_grad(ctx, a, b, g, axa, axb, fa, fb, perm, prec, wrt,
                                       Tensor.wrap(ctx, la, pa, da_data, dt) if wa else None,
                                       Tensor.wrap(ctx, lb, pb, db_data, dt) if wb else None)
                    return da_data, db_data, None

            cls._cls = Fn
        return cls._cls


def tensordot_autograd(ctx, a_data, legs_a, parity_a, b_data, legs_b, parity_b, axes_a, axes_b, flip_a=0, flip_b=0,
                       out_perm=None, prec="f64"):
    """Differentiable tensordot on flat torch CUDA tensors holding the blocks
    of A and B (block layout of the library).  Returns (C's block data, C's
    legs, C's parity); backward runs ftn_tensordot_grad."""
    spec = (ctx, [tuple(l) for l in legs_a], int(parity_a), [tuple(l) for l in legs_b], int(parity_b),
            list(axes_a), list(axes_b), int(flip_a), int(flip_b), None if out_perm is None else list(out_perm), prec)
    c = _TensordotFn.get().apply(a_data, b_data, spec)
    return c, _result_legs(spec[1], spec[3], spec[5], spec[6], spec[9]), spec[2] ^ spec[4]


class _CompressFn:
    """torch.autograd.Function over ftn_compress (forward) and
    ftn_compress_grad (backward) on flat FP64 block-data tensors (built
    lazily so that importing this module does not need torch)."""

    _cls = None

    @classmethod
    def get(cls):
        if cls._cls is None:
            import torch

            class Fn(torch.autograd.Function):
                @staticmethod
                def forward(fctx, x_data, y_data, spec):
                    ctx, lx, px, ly, py, axx, axy, chi, arrows, out = spec
                    # ftn_compress consumes its operands: it gets copies
                    x = Tensor.wrap(ctx, lx, px, x_data.detach().clone(), F64)
                    y = Tensor.wrap(ctx, ly, py, y_data.detach().clone(), F64)
                    xn, yn, info = compress(ctx, x, y, axx, axy, chi, arrows)
                    out.update(legs_x=xn.legs, parity_x=xn.parity, legs_y=yn.legs, parity_y=yn.parity, info=info)
                    fctx.save_for_backward(x_data, y_data)
                    fctx.spec = spec
                    xd, yd = xn.view().clone(), yn.view().clone()
                    ctx.synchronize()
                    return xd, yd

                @staticmethod
                def backward(fctx, gx, gy):
                    x_data, y_data = fctx.saved_tensors
                    ctx, lx, px, ly, py, axx, axy, chi, arrows, out = fctx.spec
                    x = Tensor.wrap(ctx, lx, px, x_data, F64)
                    y = Tensor.wrap(ctx, ly, py, y_data, F64)
                    nx = _numel(out["legs_x"], out["parity_x"])
                    ny = _numel(out["legs_y"], out["parity_y"])
                    gx = torch.zeros(nx, dtype=torch.float64, device=x_data.device) if gx is None else gx.contiguous()
                    gy = torch.zeros(ny, dtype=torch.float64, device=x_data.device) if gy is None else gy.contiguous()
                    dxn = Tensor.wrap(ctx, out["legs_x"], out["parity_x"], gx, F64)
                    dyn = Tensor.wrap(ctx, out["legs_y"], out["parity_y"], gy, F64)
                    dx, dy = compress_grad(ctx, x, y, axx, axy, chi, dxn, dyn, arrows)
                    dxd, dyd = dx.view().clone(), dy.view().clone()
                    ctx.synchronize()
                    return dxd, dyd, None

            cls._cls = Fn
        return cls._cls


def compress_autograd(ctx, x_data, legs_x, parity_x, y_data, legs_y, parity_y, axes_x, axes_y, chi, arrows=True):
    """Differentiable bond compression on flat FP64 torch CUDA tensors holding
    the blocks of X and Y: returns (X' data, X' legs, X' parity, Y' data, Y'
    legs, Y' parity).  Forward ftn_compress (on copies: x_data and y_data are
    left as they are), backward ftn_compress_grad."""
    out = {}
    spec = (ctx, [tuple(l) for l in legs_x], int(parity_x), [tuple(l) for l in legs_y], int(parity_y),
            list(axes_x), list(axes_y), int(chi), bool(arrows), out)
    xd, yd = _CompressFn.get().apply(x_data, y_data, spec)
    return xd, out["legs_x"], out["parity_x"], yd, out["legs_y"], out["parity_y"]


class _NetworkValueFn:
    """torch.autograd.Function for the value of a closed network of even FP64
    tensors: the forward runs ftn_contract_grad, which forms the gradient with
    the value; the backward hands it on, scaled by the incoming cotangent."""

    _cls = None

    @classmethod
    def get(cls):
        if cls._cls is None:
            import torch

            class Fn(torch.autograd.Function):
                @staticmethod
                def forward(fctx, spec, *datas):
                    ctx, legs, parities, job, checkpoint = spec
                    ts = [Tensor.wrap(ctx, lg, p, d.detach().contiguous(), F64) for lg, p, d in zip(legs, parities, datas)]
                    v, grads = contract_grad(ctx, ts, job["bonds"], job["tree"], job.get("positions"),
                                             job.get("policy", "exact"), job.get("chi", 0), checkpoint)
                    gd = [g.view().clone() for g in grads]
                    ctx.synchronize()
                    fctx.save_for_backward(*gd)
                    return torch.tensor(v, dtype=torch.float64, device=datas[0].device)

                @staticmethod
                def backward(fctx, gv):
                    return (None,) + tuple(gv * g for g in fctx.saved_tensors)

            cls._cls = Fn
        return cls._cls


def network_value_autograd(ctx, datas, legs, parities, bonds, tree, positions=None, policy="exact", chi=0,
                           checkpoint=0):
    """Differentiable value of a closed network (ftn_contract_grad) of even
    FP64 tensors given as flat torch CUDA tensors of block data with their
    legs and parities; returns a 0-dim FP64 tensor.  ``checkpoint`` as in
    contract_grad."""
    job = {"bonds": bonds, "tree": tree, "positions": positions, "policy": policy, "chi": chi}
    spec = (ctx, [[tuple(l) for l in lg] for lg in legs], [int(p) for p in parities], job, int(checkpoint))
    return _NetworkValueFn.get().apply(spec, *datas)


def transpose(ctx, t, perm, out=None):
    h = C.c_void_p(out.handle.value if out is not None else None)
    _check(lib().ftn_tensor_transpose(ctx.handle, t.handle, _int(perm), C.byref(h)))
    return out if out is not None else Tensor(ctx, h)


def dagger(ctx, t):
    h = C.c_void_p()
    _check(lib().ftn_tensor_dagger(ctx.handle, t.handle, C.byref(h)))
    return Tensor(ctx, h)


def compress(ctx, x, y, axes_x, axes_y, chi, arrows=True):
    """Returns (X', Y', info); x and y are consumed (their handles released)."""
    hx, hy = C.c_void_p(x.handle.value), C.c_void_p(y.handle.value)
    info = CompressInfo()
    _check(lib().ftn_compress(ctx.handle, C.byref(hx), C.byref(hy), len(axes_x), _int(axes_x), _int(axes_y), int(chi),
                              1 if arrows else 0, C.byref(info)))
    x.handle = None
    y.handle = None
    return Tensor(ctx, hx), Tensor(ctx, hy), info


def compress_grad(ctx, x, y, axes_x, axes_y, chi, dxn, dyn, arrows=True):
    """Gradient of a scalar of the compressed pair (ftn_compress_grad): given
    dL/dX' and dL/dY' (tensors with the legs of compress(...)'s X' and Y'),
    returns (dL/dX, dL/dY); x and y are left unchanged."""
    hx, hy = C.c_void_p(), C.c_void_p()
    _check(lib().ftn_compress_grad(ctx.handle, x.handle, y.handle, len(axes_x), _int(axes_x), _int(axes_y), int(chi),
                                   1 if arrows else 0, dxn.handle, dyn.handle, C.byref(hx), C.byref(hy)))
    return Tensor(ctx, hx), Tensor(ctx, hy)


def contract(ctx, tensors, bonds, tree, positions=None, policy="exact", chi=0, prec="f64"):
    """Contract a closed network; returns (mantissa, log_scale)."""
    arr = (C.c_void_p * len(tensors))(*[t.handle.value for t in tensors])
    flat_b = [int(v) for b in bonds for v in b]
    flat_t = [int(v) for p in tree for v in p]
    net = Network(len(tensors), C.cast(arr, C.POINTER(C.c_void_p)), len(bonds), _i32(flat_b),
                  _i32(positions) if positions is not None else None)
    tr = Tree(len(tree), _i32(flat_t), POLICY_NAMES[policy] if isinstance(policy, str) else int(policy), int(chi))
    m, lg = C.c_double(), C.c_double()
    _check(lib().ftn_contract(ctx.handle, C.byref(net), C.byref(tr), _prec(prec), C.byref(m), C.byref(lg)))
    return m.value, lg.value


def contract_grad(ctx, tensors, bonds, tree, positions=None, policy="exact", chi=0, checkpoint=0):
    """Value of a closed network of even FP64 tensors and dv/dT for every
    tensor (ftn_contract_grad): returns (value, [gradient tensors]).
    ``checkpoint`` = k > 0 keeps the walk's state every k steps and replays
    the segments in the backward (0: every intermediate kept)."""
    n, net_arr, tree_arr, keep = _network_arrays([{"tensors": tensors, "bonds": bonds, "tree": tree,
                                                   "positions": positions, "policy": policy, "chi": chi}])
    v = C.c_double()
    out = (C.c_void_p * max(1, len(tensors)))()
    _check(lib().ftn_contract_grad(ctx.handle, net_arr, tree_arr, int(checkpoint), C.byref(v), out))
    del keep
    return v.value, [Tensor(ctx, C.c_void_p(out[i])) for i in range(len(tensors))]


def _network_arrays(networks):
    """ctypes arrays of ftn_network / ftn_tree for a list of network dicts.
    The handles, bonds, trees and positions of all networks are packed into
    one flat numpy table each (the structs point into them), so packing costs
    a few vectorised copies rather than one Python conversion per integer.
    Returns (count, networks, trees, keep) -- ``keep`` holds the tables."""
    nets = list(networks)
    n = len(nets)
    if n == 0:
        return 0, (Network * 1)(), (Tree * 1)(), []

    def flat(rows):
        parts = [np.asarray(r, dtype=np.int32).reshape(-1) for r in rows]
        offs = np.zeros(len(parts) + 1, dtype=np.int64)
        np.cumsum([q.size for q in parts], out=offs[1:])
        return np.concatenate(parts + [np.zeros(1, np.int32)]), offs

    hoff = np.zeros(n + 1, dtype=np.int64)
    np.cumsum([len(job["tensors"]) for job in nets], out=hoff[1:])
    hs = np.zeros(int(hoff[-1]) + 1, dtype=np.uint64)
    hs[:-1] = np.fromiter((t.handle.value for job in nets for t in job["tensors"]), dtype=np.uint64,
                          count=int(hoff[-1]))
    fb, boff = flat(job["bonds"] for job in nets)
    ft, toff = flat(job["tree"] for job in nets)
    fp, poff = flat((() if job.get("positions") is None else job["positions"]) for job in nets)
    hp, bp, tp, pp = hs.ctypes.data, fb.ctypes.data, ft.ctypes.data, fp.ctypes.data
    # the structs themselves, filled column by column in numpy views of the
    # ctypes arrays (every pointer field is 8 bytes, every count a C int)
    nd = np.zeros(n, dtype=np.dtype({"names": ["nt", "t", "nb", "b", "p"],
                                     "formats": [np.int32, np.uint64, np.int32, np.uint64, np.uint64],
                                     "offsets": [Network.n_tensors.offset, Network.tensors.offset,
                                                 Network.n_bonds.offset, Network.bonds.offset,
                                                 Network.positions.offset],
                                     "itemsize": C.sizeof(Network)}))
    td = np.zeros(n, dtype=np.dtype({"names": ["ns", "pairs", "pol", "chi"],
                                     "formats": [np.int32, np.uint64, np.int32, np.int32],
                                     "offsets": [Tree.n_steps.offset, Tree.pairs.offset, Tree.policy.offset,
                                                 Tree.chi.offset],
                                     "itemsize": C.sizeof(Tree)}))
    has_pos = np.fromiter((job.get("positions") is not None for job in nets), dtype=bool, count=n)
    nd["nt"] = np.diff(hoff)
    nd["t"] = hp + 8 * hoff[:-1].astype(np.uint64)
    nd["nb"] = np.diff(boff) // 4
    nd["b"] = bp + 4 * boff[:-1].astype(np.uint64)
    nd["p"] = np.where(has_pos, pp + 4 * poff[:-1].astype(np.uint64), 0).astype(np.uint64)
    td["ns"] = np.diff(toff) // 2
    td["pairs"] = tp + 4 * toff[:-1].astype(np.uint64)
    pols = [job.get("policy", "exact") for job in nets]
    td["pol"] = [POLICY_NAMES[q] if isinstance(q, str) else int(q) for q in pols]
    td["chi"] = [int(job.get("chi", 0)) for job in nets]
    net_arr = (Network * n).from_buffer(nd)
    tree_arr = (Tree * n).from_buffer(td)
    return n, net_arr, tree_arr, [hs, fb, ft, fp, nd, td]


def contract_batch(ctx, networks, prec="f64"):
    """Contract many closed networks in one batched run (ftn_contract_batch).

    ``networks``: sequence of dicts with keys ``tensors``, ``bonds``, ``tree``
    and optionally ``positions``, ``policy`` ("exact") and ``chi`` (0).
    Returns a list of (mantissa, log_scale), bit-identical to :func:`contract`
    on each network alone."""
    n, net_arr, tree_arr, keep = _network_arrays(networks)
    m = (C.c_double * max(1, n))()
    lg = (C.c_double * max(1, n))()
    _check(lib().ftn_contract_batch(ctx.handle, n, net_arr, tree_arr, _prec(prec), m, lg))
    del keep
    return [(m[i], lg[i]) for i in range(n)]


def contract_batch_async(ctx, networks, d_out, prec="f64"):
    """ftn_contract_batch_async: the values of ``networks`` (as for
    :func:`contract_batch`) written on the device into ``d_out`` (a float64
    CUDA tensor of at least 2 * len(networks) elements: mantissa with its
    sign, then log-scale, per network), in stream order and without a host
    synchronisation; capturable into a CUDA graph on ctx's stream once every
    network has been contracted on this context."""
    n, net_arr, tree_arr, keep = _network_arrays(networks)
    torch = ctx._torch
    if d_out.dtype != torch.float64 or not d_out.is_cuda or not d_out.is_contiguous() or d_out.numel() < 2 * n:
        raise ValueError("d_out must be a contiguous float64 CUDA tensor of at least 2 * len(networks) elements")
    _check(lib().ftn_contract_batch_async(ctx.handle, n, net_arr, tree_arr, _prec(prec), C.c_void_p(d_out.data_ptr())))
    del keep


def _terms(num, den, group_end):
    num, den = list(num), list(den)
    ge = list(group_end) if group_end is not None else [len(num)]
    return len(num), _i32(num), _i32(den), len(ge), _i32(ge)


def energy_reduce(values, num, den, group_end=None):
    """Per-term ratios value(num[t]) / value(den[t]) and their sums per group
    (ftn_energy_reduce).  ``values``: (mantissa, log_scale) of every network.
    Returns (energies per group, ratios per term)."""
    vals = list(values)
    cnt = len(vals)
    m = (C.c_double * max(1, cnt))(*[float(v[0]) for v in vals])
    lg = (C.c_double * max(1, cnt))(*[float(v[1]) for v in vals])
    nt, fn, fd, ng, fg = _terms(num, den, group_end)
    r = (C.c_double * max(1, nt))()
    e = (C.c_double * max(1, ng))()
    _check(lib().ftn_energy_reduce(cnt, m, lg, nt, fn, fd, ng, fg, r, e))
    return [e[g] for g in range(ng)], [r[t] for t in range(nt)]


def energy(ctx, networks, num, den, group_end=None, prec="f64", batch=0):
    """Contract every network (dicts as for :func:`contract_batch`) on the
    given context(s) and reduce them to term ratios and group sums
    (ftn_energy).  ``ctx``: one Context or a list (one host thread each).
    Returns (energies per group, ratios per term, [(mantissa, log_scale)] per
    network)."""
    ctxs = list(ctx) if isinstance(ctx, (list, tuple)) else [ctx]
    carr = (C.c_void_p * len(ctxs))(*[c.handle.value for c in ctxs])
    n, net_arr, tree_arr, keep = _network_arrays(networks)
    m = (C.c_double * max(1, n))()
    lg = (C.c_double * max(1, n))()
    nt, fn, fd, ng, fg = _terms(num, den, group_end)
    r = (C.c_double * max(1, nt))()
    e = (C.c_double * max(1, ng))()
    _check(lib().ftn_energy(len(ctxs), carr, n, net_arr, tree_arr, _prec(prec), int(batch), m, lg, nt, fn, fd, ng, fg,
                            r, e))
    del keep
    return [e[g] for g in range(ng)], [r[t] for t in range(nt)], [(m[i], lg[i]) for i in range(n)]


def hubbard_term(ctx, kind, t=1.0, u=0.0, dtype=F64):
    h = C.c_void_p()
    _check(lib().ftn_hubbard_term(ctx.handle, int(kind), float(t), float(u), int(dtype), C.byref(h)))
    return Tensor(ctx, h)
