"""Python binding of the C ABI in include/ckks.h (argument marshalling only).

Every function has the name of the C entry point it wraps and raises CkksError
on a non-zero status.  Handles are small owner objects that call the matching
*_destroy when collected.  Host arrays are numpy arrays in the layouts the header
documents (coefficient domain, [limb][N] uint64).

The shared library is built in-tree by paper_2312_04356_gb300/build.py; if it is
absent, loading fails with an error (there is no fallback implementation).
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_HERE, "_build", "libckks_gb300.so")

CKKS_OK, CKKS_EINVAL, CKKS_ENOKEY, CKKS_ELEVEL, CKKS_ENOMEM, CKKS_ETIMEOUT, CKKS_ECUDA = range(7)
CKKS_SLOT, CKKS_COEFF, CKKS_CINS_REAL = 0, 1, 2
CKKS_BASIS_CHEB, CKKS_BASIS_POWER = 0, 1
CKKS_LAYER_BLOCK, CKKS_LAYER_DOWNSAMPLE = 0, 1

_lib = None


class CkksError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("ckks error %d: %s" % (code, msg))
        self.code = code


class ckks_params(ctypes.Structure):
    _fields_ = [("log_n", ctypes.c_int), ("n_q", ctypes.c_int), ("dnum", ctypes.c_int), ("n_p", ctypes.c_int),
                ("q0_bits", ctypes.c_int), ("scale_bits", ctypes.c_int), ("p_bits", ctypes.c_int),
                ("boot_bits", ctypes.c_int), ("n_boot", ctypes.c_int), ("h", ctypes.c_int),
                ("sigma", ctypes.c_double)]


class ckks_server_params(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int), ("hbm_budget", ctypes.c_longlong)]


class ckks_server_layer(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n_in", ctypes.c_int), ("n_out", ctypes.c_int), ("k", ctypes.c_int),
                ("in_index", ctypes.POINTER(ctypes.c_int)), ("convs", ctypes.POINTER(ctypes.c_void_p)),
                ("boot", ctypes.c_void_p), ("boot_in", ctypes.c_void_p)]


class ckks_boot_params(ctypes.Structure):
    _fields_ = [("w", ctypes.c_int), ("w0", ctypes.c_int), ("cout", ctypes.c_int), ("K", ctypes.c_int),
                ("r", ctypes.c_int), ("deg", ctypes.c_int), ("ctos_levels", ctypes.c_int),
                ("stoc_levels", ctypes.c_int), ("delta0", ctypes.c_double), ("stride", ctypes.c_int)]


VP = ctypes.c_void_p
PVP = ctypes.POINTER(ctypes.c_void_p)
I = ctypes.c_int
D = ctypes.c_double
U64 = ctypes.c_uint64
I64 = ctypes.c_int64

_SIGS = {
    "ckks_ctx_create": [ctypes.POINTER(ckks_params), U64, VP, PVP],
    "ckks_ctx_destroy": [VP],
    "ckks_ctx_set_allocator": [VP, VP, VP, VP],
    "ckks_ctx_pool_stats": [VP, I, VP],
    "ckks_ctx_set_inner_batching": [VP, I],
    "ckks_ctx_set_tensor_conversion": [VP, I],
    "ckks_ctx_take_device_faults": [VP, VP],
    "ckks_debug_withhold_tensor_commit": [VP, I],
    "ckks_sync": [VP],
    "ckks_ctx_info": [VP, VP, VP, VP, VP],
    "ckks_ctx_gauss_table": [VP, VP],
    "ckks_ctx_set_timing": [VP, I],
    "ckks_ctx_set_pdl": [VP, I],
    "ckks_ctx_set_side_streams": [VP, I],
    "ckks_ctx_counters": [VP, VP],
    "ckks_ctx_reset_counters": [VP],
    "ckks_ctx_kernel_stats": [VP, VP, I, VP],
    "ckks_autotune": [VP, I, VP],
    "ckks_ctx_set_ntt_variant": [VP, I],
    "ckks_ctx_set_ntt_choices": [VP, VP],
    "ckks_keygen": [VP, VP, I, I, PVP],
    "ckks_keys_add_rotations": [VP, VP, VP, I],
    "ckks_keys_destroy": [VP],
    "ckks_keys_export_secret": [VP, VP, VP],
    "ckks_ct_create": [VP, PVP],
    "ckks_ct_destroy": [VP],
    "ckks_ct_info": [VP, VP, VP],
    "ckks_ct_set_scale": [VP, D],
    "ckks_ct_import_rns": [VP, VP, I, D, VP],
    "ckks_ct_export_rns": [VP, VP, VP],
    "ckks_ct_copy_into": [VP, VP, VP],
    "ckks_pt_create": [VP, PVP],
    "ckks_pt_destroy": [VP],
    "ckks_pt_info": [VP, VP, VP],
    "ckks_pt_import_rns": [VP, VP, I, D, VP],
    "ckks_pt_export_rns": [VP, VP, VP],
    "ckks_encode": [VP, VP, VP, I, I, D, I, I, VP],
    "ckks_decode": [VP, VP, I, I, VP, VP, I],
    "ckks_encode_image": [VP, VP, I, I, I, I, D, VP],
    "ckks_decode_image": [VP, VP, I, I, I, I, VP],
    "ckks_encrypt": [VP, VP, VP, U64, VP],
    "ckks_encrypt_sk": [VP, VP, VP, U64, VP],
    "ckks_decrypt": [VP, VP, VP, VP],
    "ckks_add": [VP, VP, VP, VP],
    "ckks_sub": [VP, VP, VP, VP],
    "ckks_mul_plain": [VP, VP, VP, VP],
    "ckks_mul_relin": [VP, VP, VP, VP, VP],
    "ckks_mul_int": [VP, VP, I64, VP],
    "ckks_add_const": [VP, VP, D, VP],
    "ckks_imult": [VP, VP, VP],
    "ckks_rescale": [VP, VP, VP],
    "ckks_mod_drop": [VP, VP, I, VP],
    "ckks_level_down": [VP, VP, I, VP],
    "ckks_mod_raise": [VP, VP, VP],
    "ckks_rotate_hoisted": [VP, VP, VP, VP, I, VP],
    "ckks_conjugate": [VP, VP, VP, VP],
    "ckks_ptset_create": [VP, I, I, I, I, I, D, PVP],
    "ckks_ptset_destroy": [VP],
    "ckks_ptset_set_rns": [VP, VP, I, I, VP],
    "ckks_ptset_info": [VP, VP, VP, VP, VP, VP, VP, VP],
    "ckks_ptset_rotations": [VP, VP, I, VP],
    "ckks_bsgs": [VP, VP, VP, VP, VP],
    "ckks_ptset_conv_fused": [VP, VP, I, I, I, I, I, D, I, PVP],
    "ckks_conv2d_cins": [VP, VP, VP, VP, VP],
    "ckks_encode_dwconv_kernel": [VP, VP, I, I, I, I, D, VP],
    "ckks_ptset_conv_fused_s2": [VP, VP, I, I, I, I, I, I, D, I, PVP],
    "ckks_ptset_dwconv_fused_s2": [VP, VP, I, I, I, I, I, D, I, PVP],
    "ckks_ptset_decompose": [VP, I, I, D, I, PVP],
    "ckks_ptset_fc_stoc": [VP, VP, I, I, I, D, I, PVP],
    "ckks_fc_stoc": [VP, VP, VP, VP, I, VP],
    "ckks_boot_set_decomp": [VP, VP, VP],
    "ckks_block_multi": [VP, VP, I, PVP, PVP, VP, VP],
    "ckks_downsample_layer": [VP, VP, I, PVP, PVP, VP, PVP, VP, VP],
    "ckks_server_create": [VP, VP, ctypes.POINTER(ckks_server_params), PVP],
    "ckks_server_add_model": [VP, I, PVP, PVP, ctypes.POINTER(I)],
    "ckks_server_add_model_layers": [VP, I, ctypes.POINTER(ckks_server_layer), ctypes.POINTER(I)],
    "ckks_server_model_shape": [VP, I, VP],
    "ckks_server_model_info": [VP, I, VP],
    "ckks_server_start": [VP],
    "ckks_server_submit": [VP, I, VP, I, D, ctypes.POINTER(U64)],
    "ckks_server_poll": [VP, U64, ctypes.POINTER(I)],
    "ckks_server_wait": [VP, U64, D, ctypes.POINTER(I)],
    "ckks_server_result": [VP, U64, VP, ctypes.POINTER(I), ctypes.POINTER(D)],
    "ckks_server_cancel": [VP, U64],
    "ckks_server_stats": [VP, VP],
    "ckks_server_reset_stats": [VP],
    "ckks_server_last_error": [VP],
    "ckks_server_destroy": [VP],
    "ckks_downsample_layer_graph_create": [VP, VP, I, PVP, PVP, VP, PVP, VP, VP, PVP],
    "ckks_dwconv_cins": [VP, VP, VP, VP],
    "ckks_boot_create": [VP, ctypes.POINTER(ckks_boot_params), PVP],
    "ckks_boot_destroy": [VP],
    "ckks_boot_info": [VP, VP],
    "ckks_boot_rotations": [VP, VP, I, VP],
    "ckks_boot_bsgs_splits": [VP, VP, I, VP],
    "ckks_boot_set_bsgs_splits": [VP, VP, VP, I],
    "ckks_boot_tune_bsgs": [VP, VP, I, VP, I, VP],
    "ckks_boot_set_ctos": [VP, VP, I, VP],
    "ckks_boot_set_stoc": [VP, VP, I, VP],
    "ckks_boot_set_coeffs": [VP, VP, VP, I],
    "ckks_boot_set_masks": [VP, VP, VP, VP],
    "ckks_bootstrap": [VP, VP, VP, VP, VP, VP],
    "ckks_stoc1": [VP, VP, VP, VP, VP, VP],
    "ckks_block": [VP, VP, VP, VP, VP, VP],
    "ckks_eval_poly": [VP, VP, VP, VP, I, I, D, D, VP],
    "ckks_block_graph_create": [VP, VP, VP, VP, VP, VP, PVP],
    "ckks_graph_launch": [VP, VP],
    "ckks_graph_info": [VP, VP],
    "ckks_graph_destroy": [VP],
    "ckks_block_batch_create": [VP, VP, I, PVP, VP, VP, PVP, I, PVP],
    "ckks_batch_launch": [VP],
    "ckks_block_batched": [VP, VP, I, PVP, VP, VP, PVP],
    "ckks_block_batched_graph_create": [VP, VP, I, PVP, VP, VP, PVP, PVP],
    "ckks_downsample_layer_batched": [VP, VP, I, I, PVP, PVP, VP, PVP, VP, PVP],
    "ckks_bootstrap_batched": [VP, VP, VP, I, PVP, PVP, PVP],
    "ckks_eval_poly_batched": [VP, VP, I, PVP, VP, I, I, D, D, PVP],
    "ckks_eval_relu_batched": [VP, VP, I, PVP, VP, VP, I, PVP],
    "ckks_batch_destroy": [VP],
    "ckks_eval_relu": [VP, VP, VP, VP, VP, I, VP],
    "ckks_rescale_noalloc": [VP, VP, I, VP],
    "ckks_ntt_forward": [VP, VP, I, VP],
    "ckks_ntt_inverse": [VP, VP, I, VP],
}


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(SO_PATH):
        raise RuntimeError("CUDA library not built: %s is missing (run paper_2312_04356_gb300.build.build())"
                           % SO_PATH)
    L = ctypes.CDLL(SO_PATH)
    for name, args in _SIGS.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.ckks_last_error.argtypes = [VP]
    L.ckks_last_error.restype = ctypes.c_char_p
    L.ckks_server_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def exported_symbols():
    return list(_SIGS) + ["ckks_last_error"]


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ------------------------------------------------------------------ handles --
class _Handle:
    _destroy = None

    def __init__(self, ptr, ctx=None):
        self.ptr = ptr
        self.ctx = ctx          # keeps the context alive while the handle lives

    @property
    def _as_parameter_(self):
        return self.ptr

    def close(self):
        if self.ptr:
            getattr(lib(), self._destroy)(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context(_Handle):
    _destroy = "ckks_ctx_destroy"

    def check(self, rc):
        if rc != CKKS_OK:
            msg = lib().ckks_last_error(self.ptr)
            raise CkksError(rc, msg.decode() if msg else "")
        return rc

    def close(self):
        if self.ptr:
            lib().ckks_ctx_destroy(self.ptr)
            self.ptr = None


class Keys(_Handle):
    _destroy = "ckks_keys_destroy"


class Ciphertext(_Handle):
    _destroy = "ckks_ct_destroy"


class Plaintext(_Handle):
    _destroy = "ckks_pt_destroy"


class PtSet(_Handle):
    _destroy = "ckks_ptset_destroy"


class Boot(_Handle):
    _destroy = "ckks_boot_destroy"


class Graph(_Handle):
    _destroy = "ckks_graph_destroy"


class Batch(_Handle):
    _destroy = "ckks_batch_destroy"


class Server(_Handle):
    """the serving loop (continuous batching); keeps the objects its models use alive"""
    _destroy = "ckks_server_destroy"

    def check(self, rc):
        if rc != CKKS_OK:
            raise CkksError(rc, lib().ckks_server_last_error(self.ptr).decode())


# ------------------------------------------------------------- context ------
def ckks_ctx_create(params: dict, seed: int, stream: int = 0) -> Context:
    p = ckks_params(log_n=params["log_n"], n_q=params["n_q"], dnum=params["dnum"], n_p=params.get("n_p", 0),
                    q0_bits=params["q0_bits"], scale_bits=params["scale_bits"], p_bits=params["p_bits"],
                    boot_bits=params.get("boot_bits", 0), n_boot=params.get("n_boot", 0), h=params.get("h", 0),
                    sigma=params.get("sigma", 3.2))
    out = ctypes.c_void_p()
    rc = lib().ckks_ctx_create(ctypes.byref(p), seed, ctypes.c_void_p(stream), ctypes.byref(out))
    if rc != CKKS_OK:
        raise CkksError(rc, "context creation failed")
    ctx = Context(out.value)
    ctx.params = dict(params)
    ctx.n = 1 << params["log_n"]
    ctx.n_q = params["n_q"]
    alpha = -(-params["n_q"] // params["dnum"])
    ctx.n_p = params.get("n_p", 0) or alpha
    return ctx


def ckks_sync(ctx):
    ctx.check(lib().ckks_sync(ctx))


def ckks_ctx_info(ctx):
    q = np.zeros(ctx.n_q, dtype=np.uint64)
    p = np.zeros(ctx.n_p, dtype=np.uint64)
    psi = np.zeros(ctx.n_q + ctx.n_p, dtype=np.uint64)
    delta = np.zeros(ctx.n_q, dtype=np.float64)
    ctx.check(lib().ckks_ctx_info(ctx, _ptr(q), _ptr(p), _ptr(psi), _ptr(delta)))
    return [int(x) for x in q], [int(x) for x in p], [int(x) for x in psi], [float(x) for x in delta]


def ckks_ctx_gauss_table(ctx):
    t = np.zeros(39, dtype=np.uint64)
    ctx.check(lib().ckks_ctx_gauss_table(ctx, _ptr(t)))
    return t


def ckks_ctx_set_timing(ctx, on):
    ctx.check(lib().ckks_ctx_set_timing(ctx, int(on)))


def ckks_ctx_set_ntt_choices(ctx, choice8):
    a = np.ascontiguousarray(choice8, dtype=np.int32)
    assert a.size == 8
    ctx.check(lib().ckks_ctx_set_ntt_choices(ctx, _ptr(a)))


# caller allocator callbacks: alloc(user, bytes, stream) -> device pointer; free(user, ptr, bytes, stream)
_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


def ckks_ctx_set_allocator(ctx, alloc=None, free=None):
    """alloc(nbytes, stream) -> int device pointer (0 = out of memory), free(ptr, nbytes, stream);
    both None restores the library's stream-ordered pool.  The callback objects stay referenced
    by the context for its lifetime (buffers free through the allocator that made them)."""
    if (alloc is None) != (free is None):
        raise ValueError("give both alloc and free, or neither")
    if alloc is None:
        ctx.check(lib().ckks_ctx_set_allocator(ctx, None, None, None))
        return
    a = _ALLOC_FN(lambda user, nbytes, stream: alloc(nbytes, stream or 0) or None)
    f = _FREE_FN(lambda user, ptr, nbytes, stream: free(ptr, nbytes, stream or 0))
    if not hasattr(ctx, "_allocators"):
        ctx._allocators = []
    ctx._allocators.append((a, f))
    ctx.check(lib().ckks_ctx_set_allocator(ctx, ctypes.cast(a, VP), ctypes.cast(f, VP), None))


def torch_allocator(device=None):
    """(alloc, free) callbacks for ckks_ctx_set_allocator that serve the library from PyTorch's
    caching allocator on the stream the library names"""
    import torch
    dev = torch.cuda.current_device() if device is None else device

    def alloc(nbytes, stream):
        return torch.cuda.caching_allocator_alloc(nbytes, dev, stream)

    def free(ptr, nbytes, stream):
        torch.cuda.caching_allocator_delete(ptr)
    return alloc, free


def ckks_ctx_pool_stats(ctx, reset_high=False):
    a = np.zeros(4, dtype=np.uint64)
    ctx.check(lib().ckks_ctx_pool_stats(ctx, int(reset_high), _ptr(a)))
    return dict(zip(["used", "used_high", "reserved", "reserved_high"], [int(x) for x in a]))


def ckks_ctx_set_inner_batching(ctx, on):
    ctx.check(lib().ckks_ctx_set_inner_batching(ctx, int(on)))


def ckks_ctx_set_tensor_conversion(ctx, mode):
    ctx.check(lib().ckks_ctx_set_tensor_conversion(ctx, int(mode)))


def ckks_ctx_take_device_faults(ctx):
    a = np.zeros(1, dtype=np.uint32)
    ctx.check(lib().ckks_ctx_take_device_faults(ctx, _ptr(a)))
    return int(a[0])


def ckks_debug_withhold_tensor_commit(ctx, on):
    ctx.check(lib().ckks_debug_withhold_tensor_commit(ctx, int(on)))


def ckks_ctx_set_side_streams(ctx, on):
    ctx.check(lib().ckks_ctx_set_side_streams(ctx, int(on)))


def ckks_ctx_set_pdl(ctx, on):
    ctx.check(lib().ckks_ctx_set_pdl(ctx, int(on)))


def ckks_ctx_counters(ctx):
    a = np.zeros(6, dtype=np.int64)
    ctx.check(lib().ckks_ctx_counters(ctx, _ptr(a)))
    return dict(zip(["launches", "keyswitch", "pmult", "hrot", "hmult", "rescale"], [int(x) for x in a]))


def ckks_ctx_reset_counters(ctx):
    ctx.check(lib().ckks_ctx_reset_counters(ctx))


def ckks_ctx_kernel_stats(ctx):
    import json
    n = ctypes.c_int()
    ctx.check(lib().ckks_ctx_kernel_stats(ctx, None, 0, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value + 1)
    ctx.check(lib().ckks_ctx_kernel_stats(ctx, buf, n.value + 1, ctypes.byref(n)))
    return {k: dict(launches=int(v[0]), ms=float(v[1]), bytes=float(v[2]))
            for k, v in json.loads(buf.value.decode()).items()}


def ckks_autotune(ctx, reps=3):
    """time the NTT launch variants per limb-count class and keep the fastest"""
    a = np.zeros(8, dtype=np.int32)
    ctx.check(lib().ckks_autotune(ctx, reps, _ptr(a)))
    return [int(x) for x in a]


def ckks_ctx_set_ntt_variant(ctx, variant):
    ctx.check(lib().ckks_ctx_set_ntt_variant(ctx, variant))


# ---------------------------------------------------------------- keys ------
def ckks_keygen(ctx, rot_steps=(), want_conj=True) -> Keys:
    st = np.ascontiguousarray(list(rot_steps), dtype=np.int32)
    out = ctypes.c_void_p()
    ctx.check(lib().ckks_keygen(ctx, _ptr(st) if len(st) else None, len(st), int(want_conj), ctypes.byref(out)))
    return Keys(out.value, ctx)


def ckks_keys_add_rotations(ctx, keys, rot_steps):
    st = np.ascontiguousarray(list(rot_steps), dtype=np.int32)
    if len(st):
        ctx.check(lib().ckks_keys_add_rotations(ctx, keys, _ptr(st), len(st)))


def ckks_keys_export_secret(ctx, keys):
    s = np.zeros(ctx.n, dtype=np.int64)
    ctx.check(lib().ckks_keys_export_secret(ctx, keys, _ptr(s)))
    return s


# ------------------------------------------------------------- handles ------
def ckks_ct_create(ctx) -> Ciphertext:
    out = ctypes.c_void_p()
    ctx.check(lib().ckks_ct_create(ctx, ctypes.byref(out)))
    return Ciphertext(out.value, ctx)


def ckks_ct_info(ct):
    lev, sc = ctypes.c_int(), ctypes.c_double()
    lib().ckks_ct_info(ct, ctypes.byref(lev), ctypes.byref(sc))
    return lev.value, sc.value


def ckks_ct_set_scale(ct, scale):
    lib().ckks_ct_set_scale(ct, scale)


def ckks_ct_import_rns(ctx, limbs, level, scale, out=None):
    out = out or ckks_ct_create(ctx)
    a = _u64(limbs)
    assert a.size == 2 * (level + 1) * ctx.n
    ctx.check(lib().ckks_ct_import_rns(ctx, _ptr(a), level, scale, out))
    return out


def ckks_ct_export_rns(ctx, ct):
    lev, _ = ckks_ct_info(ct)
    a = np.zeros((2, lev + 1, ctx.n), dtype=np.uint64)
    ctx.check(lib().ckks_ct_export_rns(ctx, ct, _ptr(a)))
    return a


def ckks_ct_copy_into(ctx, src, dst):
    ctx.check(lib().ckks_ct_copy_into(ctx, src, dst))


def ckks_pt_create(ctx) -> Plaintext:
    out = ctypes.c_void_p()
    ctx.check(lib().ckks_pt_create(ctx, ctypes.byref(out)))
    return Plaintext(out.value, ctx)


def ckks_pt_info(pt):
    lev, sc = ctypes.c_int(), ctypes.c_double()
    lib().ckks_pt_info(pt, ctypes.byref(lev), ctypes.byref(sc))
    return lev.value, sc.value


def ckks_pt_import_rns(ctx, limbs, level, scale, out=None):
    out = out or ckks_pt_create(ctx)
    a = _u64(limbs)
    assert a.size == (level + 1) * ctx.n
    ctx.check(lib().ckks_pt_import_rns(ctx, _ptr(a), level, scale, out))
    return out


def ckks_pt_export_rns(ctx, pt):
    lev, _ = ckks_pt_info(pt)
    a = np.zeros((lev + 1, ctx.n), dtype=np.uint64)
    ctx.check(lib().ckks_pt_export_rns(ctx, pt, _ptr(a)))
    return a


# ------------------------------------------------------------- encoding -----
def ckks_encode(ctx, values, level, scale, kind=CKKS_SLOT, slice_len=0, out=None):
    out = out or ckks_pt_create(ctx)
    v = np.asarray(values)
    re = _f64(v.real)
    im = _f64(v.imag) if np.iscomplexobj(v) else None
    ctx.check(lib().ckks_encode(ctx, _ptr(re), _ptr(im), len(re), level, scale, kind, slice_len, out))
    return out


def ckks_decode(ctx, pt, kind=CKKS_SLOT, slice_len=0, n=None):
    if n is None:
        n = ctx.n // 2 if kind == CKKS_SLOT else ctx.n
    re = np.zeros(n, dtype=np.float64)
    im = np.zeros(n, dtype=np.float64)
    ctx.check(lib().ckks_decode(ctx, pt, kind, slice_len, _ptr(re), _ptr(im), n))
    return re + 1j * im if kind == CKKS_SLOT else re


def ckks_encode_image(ctx, img, w, level, scale, out=None):
    """img: (c, w0, w0) -> real-CinS plaintext, channel i in slice i of a w x w padded image"""
    a = _f64(img)
    c, w0 = a.shape[0], a.shape[1]
    out = out or ckks_pt_create(ctx)
    ctx.check(lib().ckks_encode_image(ctx, _ptr(a), c, w0, w, level, scale, out))
    return out


def ckks_decode_image(ctx, pt, c, w0, w, from_coeff=False):
    out = np.zeros((c, w0, w0), dtype=np.float64)
    ctx.check(lib().ckks_decode_image(ctx, pt, int(from_coeff), c, w0, w, _ptr(out)))
    return out


# ----------------------------------------------------------- encryption -----
def ckks_encrypt(ctx, keys, pt, nonce, out=None):
    out = out or ckks_ct_create(ctx)
    ctx.check(lib().ckks_encrypt(ctx, keys, pt, nonce, out))
    return out


def ckks_encrypt_sk(ctx, keys, pt, nonce, out=None):
    out = out or ckks_ct_create(ctx)
    ctx.check(lib().ckks_encrypt_sk(ctx, keys, pt, nonce, out))
    return out


def ckks_decrypt(ctx, keys, ct, out=None):
    out = out or ckks_pt_create(ctx)
    ctx.check(lib().ckks_decrypt(ctx, keys, ct, out))
    return out


# -------------------------------------------------------------- HE ops ------
def _unary(name):
    def f(ctx, ct, out=None):
        out = out or ckks_ct_create(ctx)
        ctx.check(getattr(lib(), name)(ctx, ct, out))
        return out
    f.__name__ = name
    return f


def _binary(name):
    def f(ctx, a, b, out=None):
        out = out or ckks_ct_create(ctx)
        ctx.check(getattr(lib(), name)(ctx, a, b, out))
        return out
    f.__name__ = name
    return f


ckks_add = _binary("ckks_add")
ckks_sub = _binary("ckks_sub")
ckks_mul_plain = _binary("ckks_mul_plain")
ckks_imult = _unary("ckks_imult")
ckks_rescale = _unary("ckks_rescale")
ckks_mod_raise = _unary("ckks_mod_raise")


def ckks_mul_relin(ctx, keys, a, b, out=None):
    out = out or ckks_ct_create(ctx)
    ctx.check(lib().ckks_mul_relin(ctx, keys, a, b, out))
    return out


def ckks_mul_int(ctx, ct, c, out=None):
    out = out or ckks_ct_create(ctx)
    ctx.check(lib().ckks_mul_int(ctx, ct, int(c), out))
    return out


def ckks_add_const(ctx, ct, c, out=None):
    out = out or ckks_ct_create(ctx)
    ctx.check(lib().ckks_add_const(ctx, ct, float(c), out))
    return out


def ckks_mod_drop(ctx, ct, level, out=None):
    out = out or ckks_ct_create(ctx)
    ctx.check(lib().ckks_mod_drop(ctx, ct, level, out))
    return out


def ckks_level_down(ctx, ct, level, out=None):
    out = out or ckks_ct_create(ctx)
    ctx.check(lib().ckks_level_down(ctx, ct, level, out))
    return out


def ckks_rotate_hoisted(ctx, keys, ct, steps, outs=None):
    st = np.ascontiguousarray(list(steps), dtype=np.int32)
    outs = outs or [ckks_ct_create(ctx) for _ in st]
    arr = (ctypes.c_void_p * len(outs))(*[o.ptr for o in outs])
    ctx.check(lib().ckks_rotate_hoisted(ctx, keys, ct, _ptr(st), len(st), ctypes.cast(arr, ctypes.c_void_p)))
    return outs


def ckks_conjugate(ctx, keys, ct, out=None):
    out = out or ckks_ct_create(ctx)
    ctx.check(lib().ckks_conjugate(ctx, keys, ct, out))
    return out


# ----------------------------------------------------------------- BSGS -----
def ckks_ptset_create(ctx, a0, step, count, bsgs_B, level, scale) -> PtSet:
    out = ctypes.c_void_p()
    ctx.check(lib().ckks_ptset_create(ctx, a0, step, count, bsgs_B, level, scale, ctypes.byref(out)))
    return PtSet(out.value, ctx)


def ckks_ptset_set_rns(ctx, ps, g, b, limbs):
    a = _u64(limbs)
    ctx.check(lib().ckks_ptset_set_rns(ctx, ps, g, b, _ptr(a)))


def ckks_ptset_info(ps):
    vals = [ctypes.c_int() for _ in range(5)]
    sc = ctypes.c_double()
    npts = ctypes.c_int()
    lib().ckks_ptset_info(ps, *[ctypes.byref(v) for v in vals], ctypes.byref(sc), ctypes.byref(npts))
    a0, step, count, B, level = [v.value for v in vals]
    return dict(a0=a0, step=step, count=count, B=B, level=level, scale=sc.value, n_pts=npts.value)


def ckks_ptset_rotations(ps):
    n = ctypes.c_int()
    lib().ckks_ptset_rotations(ps, None, 0, ctypes.byref(n))
    a = np.zeros(max(n.value, 1), dtype=np.int32)
    lib().ckks_ptset_rotations(ps, _ptr(a), n.value, ctypes.byref(n))
    return [int(x) for x in a[: n.value]]


def ckks_bsgs(ctx, keys, ct, ps, out=None):
    out = out or ckks_ct_create(ctx)
    ctx.check(lib().ckks_bsgs(ctx, keys, ct, ps, out))
    return out


def ckks_ptset_conv_fused(ctx, weights, cin, cout, f, w, level, pt_scale, bsgs_B=0) -> PtSet:
    W = _f64(weights)
    assert W.size == cout * cin * f * f
    out = ctypes.c_void_p()
    ctx.check(lib().ckks_ptset_conv_fused(ctx, _ptr(W), cin, cout, f, w, level, pt_scale, bsgs_B,
                                          ctypes.byref(out)))
    return PtSet(out.value, ctx)


def ckks_ptset_conv_fused_s2(ctx, weights, cin, cout, f, w_in, t, level, pt_scale, bsgs_B=0) -> PtSet:
    W = _f64(weights)
    assert W.size == cout * cin * f * f
    out = ctypes.c_void_p()
    ctx.check(lib().ckks_ptset_conv_fused_s2(ctx, _ptr(W), cin, cout, f, w_in, t, level, pt_scale, bsgs_B,
                                             ctypes.byref(out)))
    return PtSet(out.value, ctx)


def ckks_ptset_dwconv_fused_s2(ctx, K, w_in, t, level, pt_scale, bsgs_B=0) -> PtSet:
    """K: (c, f, f) stride-2 depthwise kernels -> the decomposed conv set of input ciphertext t"""
    a = _f64(K)
    assert a.ndim == 3 and a.shape[1] == a.shape[2]
    out = ctypes.c_void_p()
    ctx.check(lib().ckks_ptset_dwconv_fused_s2(ctx, _ptr(a), a.shape[0], a.shape[1], w_in, t, level, pt_scale,
                                               bsgs_B, ctypes.byref(out)))
    return PtSet(out.value, ctx)


def ckks_ptset_fc_stoc(ctx, M, level, pt_scale, bsgs_B=0) -> PtSet:
    a = _f64(M)
    n_out, n_in = a.shape
    out = ctypes.c_void_p()
    ctx.check(lib().ckks_ptset_fc_stoc(ctx, _ptr(a), n_out, n_in, level, pt_scale, bsgs_B, ctypes.byref(out)))
    return PtSet(out.value, ctx)


def ckks_fc_stoc(ctx, keys, ct, fc, n_in, out=None):
    out = out or ckks_ct_create(ctx)
    ctx.check(lib().ckks_fc_stoc(ctx, keys, ct, fc, n_in, out))
    return out


def ckks_ptset_decompose(ctx, w, level, scale, bsgs_B=0) -> PtSet:
    out = ctypes.c_void_p()
    ctx.check(lib().ckks_ptset_decompose(ctx, w, level, scale, bsgs_B, ctypes.byref(out)))
    return PtSet(out.value, ctx)


def ckks_conv2d_cins(ctx, keys, ct, conv, out=None):
    out = out or ckks_ct_create(ctx)
    ctx.check(lib().ckks_conv2d_cins(ctx, keys, ct, conv, out))
    return out


def ckks_encode_dwconv_kernel(ctx, K, w, level, scale, out=None):
    """K: (c, f, f) depthwise kernels -> one real-CinS plaintext"""
    a = _f64(K)
    out = out or ckks_pt_create(ctx)
    ctx.check(lib().ckks_encode_dwconv_kernel(ctx, _ptr(a), a.shape[0], a.shape[1], w, level, scale, out))
    return out


def ckks_dwconv_cins(ctx, ct, kernel, out=None):
    out = out or ckks_ct_create(ctx)
    ctx.check(lib().ckks_dwconv_cins(ctx, ct, kernel, out))
    return out


# -------------------------------------------------------- bootstrapping -----
def ckks_boot_create(ctx, w, w0, cout, K=28, r=3, deg=59, ctos_levels=3, stoc_levels=3, delta0=2.0 ** 49,
                     stride=1) -> Boot:
    bp = ckks_boot_params(w=w, w0=w0, cout=cout, K=K, r=r, deg=deg, ctos_levels=ctos_levels,
                          stoc_levels=stoc_levels, delta0=delta0, stride=stride)
    out = ctypes.c_void_p()
    ctx.check(lib().ckks_boot_create(ctx, ctypes.byref(bp), ctypes.byref(out)))
    return Boot(out.value, ctx)


def ckks_boot_info(bt):
    a = np.zeros(8, dtype=np.float64)
    lib().ckks_boot_info(bt, _ptr(a))
    keys = ["K_eff", "s_raise", "c_drop", "l_drop", "l_em", "l_out", "s_em", "s_mask"]
    return dict(zip(keys, [float(x) for x in a]))


def ckks_boot_rotations(bt):
    n = ctypes.c_int()
    lib().ckks_boot_rotations(bt, None, 0, ctypes.byref(n))
    a = np.zeros(max(n.value, 1), dtype=np.int32)
    lib().ckks_boot_rotations(bt, _ptr(a), n.value, ctypes.byref(n))
    return [int(x) for x in a[: n.value]]


def ckks_boot_bsgs_splits(bt):
    n = ctypes.c_int()
    a = np.zeros(64, dtype=np.int32)
    if lib().ckks_boot_bsgs_splits(bt, _ptr(a), 64, ctypes.byref(n)) != CKKS_OK:
        raise CkksError(CKKS_EINVAL, "ckks_boot_bsgs_splits")
    return [int(x) for x in a[: n.value]]


def ckks_boot_set_bsgs_splits(ctx, bt, B):
    a = np.ascontiguousarray(B, dtype=np.int32)
    ctx.check(lib().ckks_boot_set_bsgs_splits(ctx, bt, _ptr(a), len(a)))


def ckks_boot_tune_bsgs(ctx, bt, reps=3):
    n = ctypes.c_int()
    a = np.zeros(64, dtype=np.int32)
    ctx.check(lib().ckks_boot_tune_bsgs(ctx, bt, int(reps), _ptr(a), 64, ctypes.byref(n)))
    return [int(x) for x in a[: n.value]]


def ckks_boot_set_ctos(ctx, bt, i, ps):
    ctx.check(lib().ckks_boot_set_ctos(ctx, bt, i, ps))


def ckks_boot_set_stoc(ctx, bt, i, ps):
    ctx.check(lib().ckks_boot_set_stoc(ctx, bt, i, ps))


def ckks_boot_set_decomp(ctx, bt, ps):
    ctx.check(lib().ckks_boot_set_decomp(ctx, bt, ps))


def ckks_boot_set_coeffs(ctx, bt, coeffs):
    c = _f64(coeffs)
    ctx.check(lib().ckks_boot_set_coeffs(ctx, bt, _ptr(c), len(c) - 1))


def ckks_boot_set_masks(ctx, bt, re, im):
    ctx.check(lib().ckks_boot_set_masks(ctx, bt, re, im))


def ckks_bootstrap(ctx, keys, bt, ct0, out_re=None, out_im=None):
    out_re = out_re or ckks_ct_create(ctx)
    out_im = out_im or ckks_ct_create(ctx)
    ctx.check(lib().ckks_bootstrap(ctx, keys, bt, ct0, out_re, out_im))
    return out_re, out_im


def ckks_stoc1(ctx, keys, re, im, bt, out=None):
    out = out or ckks_ct_create(ctx)
    ctx.check(lib().ckks_stoc1(ctx, keys, re, im, bt, out))
    return out


def ckks_block(ctx, keys, ct, conv, bt, out=None):
    out = out or ckks_ct_create(ctx)
    ctx.check(lib().ckks_block(ctx, keys, ct, conv, bt, out))
    return out


def ckks_block_multi(ctx, keys, cts, convs, bt, out=None):
    out = out or ckks_ct_create(ctx)
    n = len(cts)
    assert n == len(convs)
    a = (ctypes.c_void_p * n)(*[c.ptr for c in cts])
    b = (ctypes.c_void_p * n)(*[c.ptr for c in convs])
    ctx.check(lib().ckks_block_multi(ctx, keys, n, a, b, bt, out))
    return out


def _ptrs(hs):
    return (ctypes.c_void_p * len(hs))(*[h.ptr for h in hs])


def ckks_downsample_layer(ctx, keys, res, ims, bt_in, convs, bt_out, out=None):
    out = out or ckks_ct_create(ctx)
    n = len(res)
    assert n == len(ims) == len(convs)
    ctx.check(lib().ckks_downsample_layer(ctx, keys, n, _ptrs(res), _ptrs(ims), bt_in, _ptrs(convs), bt_out, out))
    return out


def ckks_downsample_layer_graph_create(ctx, keys, res, ims, bt_in, convs, bt_out, out) -> "Graph":
    n = len(res)
    assert n == len(ims) == len(convs)
    g = ctypes.c_void_p()
    ctx.check(lib().ckks_downsample_layer_graph_create(ctx, keys, n, _ptrs(res), _ptrs(ims), bt_in, _ptrs(convs),
                                                       bt_out, out, ctypes.byref(g)))
    gr = Graph(g.value, ctx)
    gr.refs = (keys, list(res), list(ims), bt_in, list(convs), bt_out, out)
    return gr


def ckks_block_graph_create(ctx, keys, ct, conv, bt, out) -> Graph:
    g = ctypes.c_void_p()
    ctx.check(lib().ckks_block_graph_create(ctx, keys, ct, conv, bt, out, ctypes.byref(g)))
    gr = Graph(g.value, ctx)
    gr.refs = (keys, ct, conv, bt, out)     # the graph reads and writes these buffers
    return gr


def ckks_block_batch_create(ctx, keys, ins, conv, bt, outs, n_streams=8) -> Batch:
    """one block graph per input (ins[i] -> outs[i]) over n_streams streams of the batch's own"""
    n = len(ins)
    assert n == len(outs)
    b = ctypes.c_void_p()
    ctx.check(lib().ckks_block_batch_create(ctx, keys, n, _ptrs(ins), conv, bt, _ptrs(outs), n_streams,
                                            ctypes.byref(b)))
    bh = Batch(b.value, ctx)
    bh.refs = (keys, list(ins), conv, bt, list(outs))     # the graphs read and write these buffers
    return bh


def ckks_block_batched(ctx, keys, ins, conv, bt, outs=None):
    """the lockstep batch: every input through one block, each kernel launched once for all"""
    outs = outs or [ckks_ct_create(ctx) for _ in ins]
    assert len(outs) == len(ins)
    ctx.check(lib().ckks_block_batched(ctx, keys, len(ins), _ptrs(ins), conv, bt, _ptrs(outs)))
    return outs


def ckks_downsample_layer_batched(ctx, keys, res, ims, bt_in, convs, bt_out, outs=None):
    """res[b][t], ims[b][t]: input b's n_in EvalMod output pairs; one lockstep batch over b"""
    B, n_in = len(res), len(convs)
    assert all(len(r) == n_in for r in res) and all(len(i) == n_in for i in ims) and len(ims) == B
    outs = outs or [ckks_ct_create(ctx) for _ in range(B)]
    flat_r = [c for r in res for c in r]
    flat_i = [c for i in ims for c in i]
    ctx.check(lib().ckks_downsample_layer_batched(ctx, keys, B, n_in, _ptrs(flat_r), _ptrs(flat_i), bt_in,
                                                  _ptrs(convs), bt_out, _ptrs(outs)))
    return outs


def ckks_bootstrap_batched(ctx, keys, bt, ins):
    re = [ckks_ct_create(ctx) for _ in ins]
    im = [ckks_ct_create(ctx) for _ in ins]
    ctx.check(lib().ckks_bootstrap_batched(ctx, keys, bt, len(ins), _ptrs(ins), _ptrs(re), _ptrs(im)))
    return re, im


def ckks_eval_poly_batched(ctx, keys, ins, coeffs, basis=CKKS_BASIS_CHEB, a=-1.0, b=1.0):
    outs = [ckks_ct_create(ctx) for _ in ins]
    c = _f64(coeffs)
    ctx.check(lib().ckks_eval_poly_batched(ctx, keys, len(ins), _ptrs(ins), _ptr(c), len(c) - 1, basis, a, b,
                                           _ptrs(outs)))
    return outs


def ckks_eval_relu_batched(ctx, keys, ins, stages):
    outs = [ckks_ct_create(ctx) for _ in ins]
    c = _f64(np.concatenate([np.asarray(st, dtype=np.float64) for st in stages]))
    degs = np.ascontiguousarray([len(st) - 1 for st in stages], dtype=np.int32)
    ctx.check(lib().ckks_eval_relu_batched(ctx, keys, len(ins), _ptrs(ins), _ptr(c), _ptr(degs), len(stages),
                                           _ptrs(outs)))
    return outs


def ckks_block_batched_graph_create(ctx, keys, ins, conv, bt, outs) -> Graph:
    assert len(outs) == len(ins)
    g = ctypes.c_void_p()
    ctx.check(lib().ckks_block_batched_graph_create(ctx, keys, len(ins), _ptrs(ins), conv, bt, _ptrs(outs),
                                                    ctypes.byref(g)))
    gr = Graph(g.value, ctx)
    gr.refs = (keys, list(ins), conv, bt, list(outs))     # the graph reads and writes these buffers
    return gr


def ckks_batch_launch(batch):
    batch.ctx.check(lib().ckks_batch_launch(batch))


def ckks_graph_launch(graph, stream=0):
    graph.ctx.check(lib().ckks_graph_launch(graph, ctypes.c_void_p(stream)))


def ckks_graph_info(graph):
    n = ctypes.c_int64()
    lib().ckks_graph_info(graph, ctypes.byref(n))
    return n.value


def ckks_eval_poly(ctx, keys, ct, coeffs, basis=CKKS_BASIS_CHEB, a=-1.0, b=1.0, out=None):
    out = out or ckks_ct_create(ctx)
    c = _f64(coeffs)
    ctx.check(lib().ckks_eval_poly(ctx, keys, ct, _ptr(c), len(c) - 1, basis, a, b, out))
    return out


def ckks_eval_relu(ctx, keys, ct, stages, out=None):
    """composite polynomial ReLU: stages = list of Chebyshev coefficient lists"""
    out = out or ckks_ct_create(ctx)
    c = _f64(np.concatenate([np.asarray(s, dtype=np.float64) for s in stages]))
    degs = np.ascontiguousarray([len(s) - 1 for s in stages], dtype=np.int32)
    ctx.check(lib().ckks_eval_relu(ctx, keys, ct, _ptr(c), _ptr(degs), len(stages), out))
    return out


# --------------------------------------------- rescale without allocation ---
def ckks_rescale_noalloc(ctx, d_in, level, d_out):
    """rescale of raw device arrays ([2][level+1][N] -> [2][level][N], NTT domain) using the
    library's static scratch array instead of allocating (see include/ckks.h)"""
    ctx.check(lib().ckks_rescale_noalloc(ctx, ctypes.c_void_p(d_in), level, ctypes.c_void_p(d_out)))


# ------------------------------------------------------------- raw NTT ------
def ckks_ntt_forward(ctx, dev_ptr, n_limbs, prime_ids):
    ids = np.ascontiguousarray(prime_ids, dtype=np.int32)
    ctx.check(lib().ckks_ntt_forward(ctx, ctypes.c_void_p(dev_ptr), n_limbs, _ptr(ids)))


def ckks_ntt_inverse(ctx, dev_ptr, n_limbs, prime_ids):
    ids = np.ascontiguousarray(prime_ids, dtype=np.int32)
    ctx.check(lib().ckks_ntt_inverse(ctx, ctypes.c_void_p(dev_ptr), n_limbs, _ptr(ids)))


# ------------------------------------------------------------- serving loop -----
CKKS_REQ_QUEUED, CKKS_REQ_RUNNING, CKKS_REQ_DONE, CKKS_REQ_FAILED, CKKS_REQ_CANCELLED = range(5)


def ckks_server_create(ctx, keys, slots, hbm_budget=0) -> Server:
    sp = ckks_server_params(slots=slots, hbm_budget=int(hbm_budget))
    out = ctypes.c_void_p()
    ctx.check(lib().ckks_server_create(ctx, keys, ctypes.byref(sp), ctypes.byref(out)))
    srv = Server(out.value, ctx)
    srv.refs = [keys]
    return srv


def ckks_server_add_model(srv, convs, boots):
    n = len(convs)
    assert n == len(boots)
    mid = ctypes.c_int()
    srv.check(lib().ckks_server_add_model(srv, n, _ptrs(convs), _ptrs(boots), ctypes.byref(mid)))
    srv.refs += list(convs) + list(boots)
    return mid.value


def ckks_server_add_model_layers(srv, layers):
    """layers: dicts with kind (CKKS_LAYER_BLOCK / CKKS_LAYER_DOWNSAMPLE), convs (n_out lists of
    k sets, output-major), boot, for a downsampling layer boot_in, and optionally inputs (n_out
    lists of k input indices, with n_in the number of inputs; default: every output reads all)"""
    arr = (ckks_server_layer * len(layers))()
    keep = []
    for k, L in enumerate(layers):
        rows = L["convs"]
        flat = [p for row in rows for p in row]
        cv = _ptrs(flat)
        keep.append(cv)
        arr[k].kind = L["kind"]
        arr[k].k = len(rows[0])
        arr[k].n_out = len(rows)
        if L.get("inputs") is not None:
            idx = (ctypes.c_int * (len(rows) * len(rows[0])))(*[i for row in L["inputs"] for i in row])
            keep.append(idx)
            arr[k].in_index = ctypes.cast(idx, ctypes.POINTER(ctypes.c_int))
            arr[k].n_in = L["n_in"]
        else:
            arr[k].n_in = len(rows[0])
        arr[k].convs = ctypes.cast(cv, ctypes.POINTER(ctypes.c_void_p))
        arr[k].boot = L["boot"].ptr
        arr[k].boot_in = L["boot_in"].ptr if L.get("boot_in") is not None else None
        srv.refs += flat + [L["boot"]] + ([L["boot_in"]] if L.get("boot_in") is not None else [])
    mid = ctypes.c_int()
    srv.check(lib().ckks_server_add_model_layers(srv, len(layers), arr, ctypes.byref(mid)))
    return mid.value


def ckks_server_model_shape(srv, model_id):
    a = np.zeros(2, dtype=np.int32)
    srv.check(lib().ckks_server_model_shape(srv, model_id, _ptr(a)))
    return int(a[0]), int(a[1])


def ckks_server_model_info(srv, model_id):
    a = np.zeros(6, dtype=np.float64)
    srv.check(lib().ckks_server_model_info(srv, model_id, _ptr(a)))
    keys = ["in_level", "in_scale", "out_level", "out_scale", "footprint", "kernels"]
    return dict(zip(keys, [float(x) for x in a]))


def ckks_server_start(srv):
    srv.check(lib().ckks_server_start(srv))


def ckks_server_submit(srv, model_id, limbs, level, scale):
    a = np.ascontiguousarray(limbs, dtype=np.uint64)
    rid = ctypes.c_uint64()
    srv.check(lib().ckks_server_submit(srv, model_id, _ptr(a), level, scale, ctypes.byref(rid)))
    return rid.value


def ckks_server_poll(srv, rid):
    st = ctypes.c_int()
    srv.check(lib().ckks_server_poll(srv, rid, ctypes.byref(st)))
    return st.value


def ckks_server_wait(srv, rid, timeout_s=60.0):
    st = ctypes.c_int()
    rc = lib().ckks_server_wait(srv, rid, timeout_s, ctypes.byref(st))
    if rc not in (CKKS_OK, CKKS_ETIMEOUT):
        srv.check(rc)
    return st.value


def ckks_server_result(srv, rid, n, n_out=1):
    """limbs [2][level + 1][N] of a one-output model, [n_out][2][level + 1][N] otherwise"""
    lev, sc = ctypes.c_int(), ctypes.c_double()
    srv.check(lib().ckks_server_result(srv, rid, None, ctypes.byref(lev), ctypes.byref(sc)))
    out = np.zeros((2, lev.value + 1, n) if n_out == 1 else (n_out, 2, lev.value + 1, n), dtype=np.uint64)
    srv.check(lib().ckks_server_result(srv, rid, _ptr(out), ctypes.byref(lev), ctypes.byref(sc)))
    return out, lev.value, sc.value


def ckks_server_cancel(srv, rid):
    srv.check(lib().ckks_server_cancel(srv, rid))


def ckks_server_stats(srv):
    a = np.zeros(8, dtype=np.float64)
    srv.check(lib().ckks_server_stats(srv, _ptr(a)))
    keys = ["completed", "failed", "cancelled", "p50_ms", "p99_ms", "mean_ms", "max_in_flight", "kernels"]
    return dict(zip(keys, [float(x) for x in a]))


def ckks_server_reset_stats(srv):
    srv.check(lib().ckks_server_reset_stats(srv))
