"""Loader for the oracle's C primitives (oracle/ckks_ref.c).

TEST INFRASTRUCTURE ONLY: the oracle checks the CUDA library and is never on its
path.  Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline and
reference legs may import anything under oracle/.

The shared object is compiled with plain gcc (-O2 -fopenmp) into oracle/_build/.
Every wrapper takes and returns C-contiguous numpy uint64 arrays laid out
[limb][coefficient].
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ckks_ref.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libckks_ref.so")
_lock = threading.Lock()
_lib = None

U64P = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
I64P = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
I32P = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
u64 = ctypes.c_uint64
c_int = ctypes.c_int


def build(force=False):
    """Compile the oracle shared object (gcc, no CUDA)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        L = ctypes.CDLL(_SO)
        sig = {
            "orc_pow_mod": (u64, [u64, u64, u64]),
            "orc_mul_mod": (u64, [u64, u64, u64]),
            "orc_max_threads": (c_int, []),
            "orc_set_threads": (None, [c_int]),
            "orc_ntt_naive": (None, [U64P, U64P, c_int, u64, u64]),
            "orc_ntt_forward": (None, [U64P, c_int, c_int, U64P, U64P]),
            "orc_ntt_inverse": (None, [U64P, c_int, c_int, U64P, U64P]),
            "orc_negacyclic_naive": (None, [U64P, U64P, U64P, c_int, u64]),
            "orc_add": (None, [U64P, U64P, U64P, c_int, c_int, U64P]),
            "orc_sub": (None, [U64P, U64P, U64P, c_int, c_int, U64P]),
            "orc_neg": (None, [U64P, U64P, c_int, c_int, U64P]),
            "orc_mul": (None, [U64P, U64P, U64P, c_int, c_int, U64P]),
            "orc_mul_acc": (None, [U64P, U64P, U64P, c_int, c_int, U64P]),
            "orc_mul_scalar": (None, [U64P, U64P, U64P, c_int, c_int, U64P]),
            "orc_signed_to_rns": (None, [I64P, U64P, c_int, c_int, U64P]),
            "orc_automorphism": (None, [U64P, U64P, c_int, c_int, U64P, u64]),
            "orc_base_convert": (None, [U64P, c_int, U64P, U64P, c_int, U64P, c_int]),
            "orc_rescale": (None, [U64P, U64P, c_int, c_int, U64P]),
            "orc_mod_down": (None, [U64P, U64P, c_int, c_int, c_int, U64P, U64P]),
            "orc_div_round": (None, [U64P, U64P, c_int, c_int, c_int, U64P, U64P]),
            "orc_mod_raise": (None, [U64P, U64P, c_int, c_int, U64P]),
            "orc_splitmix_mix": (u64, [u64]),
            "orc_stream_key": (u64, [u64, u64]),
            "orc_stream_word": (u64, [u64, u64]),
            "orc_sample_uniform": (None, [U64P, c_int, c_int, U64P, I32P, u64, u64]),
            "orc_sample_ternary": (None, [I64P, c_int, u64, u64]),
            "orc_sample_hw": (None, [I64P, c_int, c_int, u64, u64, u64]),
            "orc_gauss_table": (None, [ctypes.c_double, U64P]),
            "orc_sample_gauss": (None, [I64P, c_int, ctypes.c_double, u64, u64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def _u(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def _mods(q):
    return np.ascontiguousarray(np.asarray(q, dtype=np.uint64))


# ---- thin numpy wrappers -------------------------------------------------

def ntt_forward(a, q, psi, logn):
    a = _u(a).copy()
    lib().orc_ntt_forward(a, a.shape[0], logn, _mods(q), _mods(psi))
    return a


def ntt_inverse(a, q, psi, logn):
    a = _u(a).copy()
    lib().orc_ntt_inverse(a, a.shape[0], logn, _mods(q), _mods(psi))
    return a


def ntt_naive(a, q, psi, logn):
    a = _u(a)
    out = np.zeros_like(a)
    lib().orc_ntt_naive(a, out, logn, int(q), int(psi))
    return out


def negacyclic_naive(a, b, q):
    a, b = _u(a), _u(b)
    out = np.zeros_like(a)
    lib().orc_negacyclic_naive(a, b, out, a.shape[0], int(q))
    return out


def _binop(name, a, b, q):
    a, b = _u(a), _u(b)
    out = np.empty_like(a)
    getattr(lib(), name)(a, b, out, a.shape[0], a.shape[1], _mods(q))
    return out


def add(a, b, q):
    return _binop("orc_add", a, b, q)


def sub(a, b, q):
    return _binop("orc_sub", a, b, q)


def mul(a, b, q):
    return _binop("orc_mul", a, b, q)


def mul_acc(acc, a, b, q):
    """acc += a*b (pointwise), in place on acc."""
    a, b = _u(a), _u(b)
    lib().orc_mul_acc(a, b, acc, a.shape[0], a.shape[1], _mods(q))
    return acc


def neg(a, q):
    a = _u(a)
    out = np.empty_like(a)
    lib().orc_neg(a, out, a.shape[0], a.shape[1], _mods(q))
    return out


def mul_scalar(a, s, q):
    """a * s[limb], s a per-limb residue vector."""
    a = _u(a)
    out = np.empty_like(a)
    lib().orc_mul_scalar(a, _mods(s), out, a.shape[0], a.shape[1], _mods(q))
    return out


def signed_to_rns(v, q):
    v = np.ascontiguousarray(v, dtype=np.int64)
    out = np.empty((len(q), v.shape[0]), dtype=np.uint64)
    lib().orc_signed_to_rns(v, out, len(q), v.shape[0], _mods(q))
    return out


def automorphism(a, q, g, logn):
    a = _u(a)
    out = np.empty_like(a)
    lib().orc_automorphism(a, out, a.shape[0], logn, _mods(q), int(g))
    return out


def base_convert(x, qin, qout):
    x = _u(x)
    out = np.empty((len(qout), x.shape[1]), dtype=np.uint64)
    lib().orc_base_convert(x, len(qin), _mods(qin), out, len(qout), _mods(qout), x.shape[1])
    return out


def rescale(c, q):
    """c: [l+1][n] over q[0..l] -> [l][n]."""
    c = _u(c)
    l = c.shape[0] - 1
    out = np.empty((l, c.shape[1]), dtype=np.uint64)
    lib().orc_rescale(c, out, l, c.shape[1], _mods(q[: l + 1]))
    return out


def mod_down(c, q, p):
    c = _u(c)
    nq, np_ = len(q), len(p)
    out = np.empty((nq, c.shape[1]), dtype=np.uint64)
    lib().orc_mod_down(c, out, nq, np_, c.shape[1], _mods(q), _mods(p))
    return out


def div_round(x, level, q, S):
    """x: rows q_0..q_{level-1} then one row per modulus of S ([level + len(S)][n]) ->
    round(x / prod S) over q_0..q_{level-1} ([level][n]), exact"""
    x = _u(x)
    out = np.empty((level, x.shape[1]), dtype=np.uint64)
    lib().orc_div_round(x, out, level, len(S), x.shape[1], _mods(q[:level]), _mods(S))
    return out


def mod_raise(c0, q):
    c0 = _u(c0).reshape(1, -1)
    out = np.empty((len(q), c0.shape[1]), dtype=np.uint64)
    lib().orc_mod_raise(c0, out, len(q), c0.shape[1], _mods(q))
    return out


def sample_uniform(q, prime_ids, n, seed, tag):
    out = np.empty((len(q), n), dtype=np.uint64)
    lib().orc_sample_uniform(out, len(q), n, _mods(q),
                             np.ascontiguousarray(prime_ids, dtype=np.int32), seed, tag)
    return out


def sample_ternary(n, seed, tag):
    out = np.empty(n, dtype=np.int64)
    lib().orc_sample_ternary(out, n, seed, tag)
    return out


def sample_hw(n, h, seed, tag_pos, tag_sign):
    out = np.empty(n, dtype=np.int64)
    lib().orc_sample_hw(out, n, h, seed, tag_pos, tag_sign)
    return out


def gauss_table(sigma):
    t = np.zeros(39, dtype=np.uint64)
    lib().orc_gauss_table(sigma, t)
    return t


def sample_gauss(n, sigma, seed, tag):
    out = np.empty(n, dtype=np.int64)
    lib().orc_sample_gauss(out, n, sigma, seed, tag)
    return out


def max_threads():
    """threads of the oracle's OpenMP loops"""
    return int(lib().orc_max_threads())


def set_threads(n):
    """use n threads in the oracle's OpenMP loops from now on"""
    lib().orc_set_threads(int(n))


def splitmix_mix(z):
    return int(lib().orc_splitmix_mix(z))


def stream_key(seed, tag):
    return int(lib().orc_stream_key(seed, tag))


def stream_word(key, i):
    return int(lib().orc_stream_word(key, i))
