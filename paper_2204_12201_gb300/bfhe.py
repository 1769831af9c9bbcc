"""Thin Python binding of the bfhe C ABI (include/bfhe.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Buffers are torch int64 tensors on the context's CUDA device
(residues < 2^60, so the bit patterns equal the ABI's uint64 words); calls
are asynchronous on torch's current stream.  The library must be built
(``paper_2204_12201_gb300.build.build()``); there is no CPU fallback and a
missing library raises.
"""

import ctypes
import os

import torch

from .build import lib_path

AND, OR, XOR, NAND, NOR, XNOR, NOT, MUX = range(8)
OP_MUL, OP_LIN = 8, 9
PAPER, SELECT = 0, 1
KERNEL_CLASSES = ("ntt_fwd", "ntt_inv", "modup", "tensor", "scale", "inner", "moddown")

_lib = None


class BfheError(RuntimeError):
    pass


def load():
    """Load libbfhe.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise BfheError("libbfhe.so not built: run paper_2204_12201_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, S, U32, U64, I = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    sig = {
        "bfhe_ctx_create": (I, [P, I, P]),
        "bfhe_param_primes": (I, [P, P, P]),
        "bfhe_ctx_destroy": (None, [P]),
        "bfhe_ctx_primes": (I, [P, P, P]),
        "bfhe_reserve": (I, [P, S]),
        "bfhe_ctx_device_bytes": (I, [P, P]),
        "bfhe_mul_scratch_bytes": (S, [P, S]),
        "bfhe_keygen": (I, [P, U64, P]),
        "bfhe_export_keys": (I, [P, P, P, P, P]),
        "bfhe_encrypt": (I, [P, P, S, U64, P, P]),
        "bfhe_decrypt": (I, [P, P, S, P, P]),
        "bfhe_add": (I, [P, P, P, P, S, P]),
        "bfhe_sub": (I, [P, P, P, P, S, P]),
        "bfhe_add_const": (I, [P, P, U64, P, S, P]),
        "bfhe_sub_const": (I, [P, P, U64, P, S, P]),
        "bfhe_const_sub": (I, [P, U64, P, P, S, P]),
        "bfhe_mul_scalar": (I, [P, P, U64, P, S, P]),
        "bfhe_mul_plain": (I, [P, P, P, P, S, P]),
        "bfhe_mul_relin": (I, [P, P, P, P, S, P]),
        "bfhe_mul_relin_noalloc": (I, [P, P, P, P, S, P]),
        "bfhe_bit_gate": (I, [P, I, P, P, P, P, S, P]),
        "bfhe_gate_level": (I, [P, P, S, S, P, S, S, P]),
        "bfhe_bits_to_mod": (I, [P, P, U32, P, S, P]),
        "bfhe_mod_to_bits": (I, [P, P, U32, U64, U64, I, P, S, P]),
        "bfhe_sint_to_mod": (I, [P, P, U32, P, S, P]),
        "bfhe_encrypt_poly": (I, [P, P, S, U64, P, P]),
        "bfhe_decrypt_poly": (I, [P, P, S, P, P]),
        "bfhe_mod_to_sint": (I, [P, P, U32, U64, U64, U64, U64, I, P, S, P]),
        "bfhe_pow": (I, [P, P, U64, P, S, P]),
        "bfhe_op_counts": (I, [P, P, I]),
        "bfhe_ntt": (I, [P, P, S, U32, I, P]),
        "bfhe_profile": (I, [P, I]),
        "bfhe_profile_read": (I, [P, P, P, P, P]),
        "bfhe_probe_modmul": (I, [I, U32, P, P]),
        "bfhe_launch_count": (ctypes.c_uint64, []),
        "bfhe_set_scratch_budget": (I, [S]),
        "bfhe_check": (I, [P, P, P]),
        "bfhe_set_fast_extension": (I, [P, I]),
        "bfhe_fast_extension": (I, [P]),
        "bfhe_set_graph_tiles": (I, [P, I]),
        "bfhe_graph_tiles": (I, [P]),
        "bfhe_scratch_budget": (S, []),
        "bfhe_set_mul_tile": (I, [U32, S]),
        "bfhe_mul_tile": (S, [U32]),
        "bfhe_ntt_config": (I, [U32, I, U32, U32, P, P]),
        "bfhe_strerror": (ctypes.c_char_p, [I]),
        "bfhe_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class _Params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_uint32), ("L", ctypes.c_uint32), ("alpha", ctypes.c_uint32),
                ("prime_bits", ctypes.c_uint32), ("t", ctypes.c_uint64)]


def _check(rc):
    if rc != 0:
        lib = load()
        raise BfheError("%s (%d): %s" % (lib.bfhe_strerror(rc).decode(), rc, lib.bfhe_last_error().decode()))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Context:
    """One parameter set, its keys and its scratch, on one CUDA device."""

    def __init__(self, N, L, alpha, t=65537, prime_bits=50, device=0):
        self.lib = load()
        self.N, self.L, self.alpha, self.t = N, L, alpha, t
        self.device = torch.device("cuda", device)
        prm = _Params(N, L, alpha, prime_bits, t)
        h = ctypes.c_void_p()
        torch.cuda.set_device(device)
        _check(self.lib.bfhe_ctx_create(ctypes.byref(prm), device, ctypes.byref(h)))
        self.h = h
        buf = (ctypes.c_uint64 * 80)()
        K = ctypes.c_uint32()
        _check(self.lib.bfhe_ctx_primes(self.h, buf, ctypes.byref(K)))
        self.K = K.value
        self.primes = [int(buf[i]) for i in range(L + alpha + self.K)]

    def close(self):
        if getattr(self, "h", None):
            torch.cuda.synchronize(self.device)
            self.lib.bfhe_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- helpers
    @property
    def stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def empty_ct(self, n, *lead):
        return torch.empty(*lead, n, 2, self.L, self.N, dtype=torch.int64, device=self.device)

    def _n(self, ct):
        assert ct.dtype == torch.int64 and ct.is_cuda and ct.is_contiguous()
        assert ct.shape[-3:] == (2, self.L, self.N), ct.shape
        return ct.numel() // (2 * self.L * self.N)

    # ---------------------------------------------------------------- ABI
    def check(self):
        """Synchronise the current stream; raise BfheError if a kernel saw an out-of-range input
        since the previous check (flags BFHE_FLAG_PLAINTEXT = 1, BFHE_FLAG_RESIDUE = 2)."""
        f = ctypes.c_uint32(0)
        rc = self.lib.bfhe_check(self.h, self.stream, ctypes.byref(f))
        if rc != 0 and f.value == 0:
            _check(rc)
        if f.value:
            err = BfheError("out-of-range input (flags %d): %s" % (f.value, self.lib.bfhe_last_error().decode()))
            err.flags = f.value
            raise err

    def set_fast_extension(self, on):
        """Guarded fast base extension in the multiply (same results, different speed)."""
        _check(self.lib.bfhe_set_fast_extension(self.h, int(bool(on))))

    @property
    def fast_extension(self):
        rc = self.lib.bfhe_fast_extension(self.h)
        if rc < 0:
            _check(rc)
        return bool(rc)

    def set_graph_tiles(self, on):
        """mod_to_bits replays its full candidate tiles from one captured CUDA graph (same results)."""
        _check(self.lib.bfhe_set_graph_tiles(self.h, int(bool(on))))

    @property
    def graph_tiles(self):
        rc = self.lib.bfhe_graph_tiles(self.h)
        if rc < 0:
            _check(rc)
        return bool(rc)

    def reserve(self, n):
        _check(self.lib.bfhe_reserve(self.h, n))

    def device_bytes(self):
        """{tables, keys, scratch, other}: device memory the context holds (bytes)."""
        out = (ctypes.c_size_t * 4)()
        _check(self.lib.bfhe_ctx_device_bytes(self.h, out))
        return {"tables": out[0], "keys": out[1], "scratch": out[2], "other": out[3]}

    def mul_scratch_bytes(self, n):
        """Scratch one mul_relin of n ciphertexts uses."""
        return int(self.lib.bfhe_mul_scratch_bytes(self.h, n))

    def keygen(self, seed):
        _check(self.lib.bfhe_keygen(self.h, seed, self.stream))

    def export_keys(self):
        sk = torch.empty(self.N, dtype=torch.int64, device=self.device)
        pk = torch.empty(2, self.L, self.N, dtype=torch.int64, device=self.device)
        rlk = torch.empty(self.L, 2, self.L + self.alpha, self.N, dtype=torch.int64, device=self.device)
        _check(self.lib.bfhe_export_keys(self.h, _ptr(sk), _ptr(pk), _ptr(rlk), self.stream))
        return sk, pk, rlk

    def encrypt(self, slots, seed, out=None):
        slots = slots.contiguous()
        n = slots.numel() // self.N
        out = self.empty_ct(n) if out is None else out
        _check(self.lib.bfhe_encrypt(self.h, _ptr(slots), n, seed, _ptr(out), self.stream))
        return out

    @property
    def batching(self):
        """False at t = 2: coefficient encoding only (encrypt_poly / decrypt_poly)."""
        return self.t != 2

    def encrypt_poly(self, coeffs, seed, out=None):
        """coeffs [n][N] plaintext polynomials (coefficients < t)."""
        coeffs = coeffs.contiguous()
        n = coeffs.numel() // self.N
        out = self.empty_ct(n) if out is None else out
        _check(self.lib.bfhe_encrypt_poly(self.h, _ptr(coeffs), n, seed, _ptr(out), self.stream))
        return out

    def decrypt_poly(self, ct, out=None):
        n = self._n(ct)
        out = torch.empty(n, self.N, dtype=torch.int64, device=self.device) if out is None else out
        _check(self.lib.bfhe_decrypt_poly(self.h, _ptr(ct), n, _ptr(out), self.stream))
        return out

    def decrypt(self, ct, out=None):
        n = self._n(ct)
        out = torch.empty(n, self.N, dtype=torch.int64, device=self.device) if out is None else out
        _check(self.lib.bfhe_decrypt(self.h, _ptr(ct), n, _ptr(out), self.stream))
        return out

    def _same(self, n, *cts):
        """Every buffer holds n ciphertexts (checked before the library reads or writes them)."""
        for c in cts:
            if c is not None and self._n(c) != n:
                raise ValueError("batch sizes differ: %d vs %d ciphertexts" % (self._n(c), n))

    def _binary(self, fn, a, b, out):
        n = self._n(a)
        out = torch.empty_like(a) if out is None else out
        self._same(n, b, out)
        _check(fn(self.h, _ptr(a), _ptr(b), _ptr(out), n, self.stream))
        return out

    def add(self, a, b, out=None):
        return self._binary(self.lib.bfhe_add, a, b, out)

    def sub(self, a, b, out=None):
        return self._binary(self.lib.bfhe_sub, a, b, out)

    def mul_relin(self, a, b, out=None):
        return self._binary(self.lib.bfhe_mul_relin, a, b, out)

    def mul_relin_noalloc(self, a, b, out=None):
        """bfhe_mul_relin_noalloc: same product, scratch in the library's static device array."""
        return self._binary(self.lib.bfhe_mul_relin_noalloc, a, b, out)

    def mul_plain(self, a, plain, out=None):
        n = self._n(a)
        plain = plain.contiguous()
        if plain.numel() != n * self.N:
            raise ValueError("plain holds %d words, want %d slot vectors of %d" % (plain.numel(), n, self.N))
        out = torch.empty_like(a) if out is None else out
        self._same(n, out)
        _check(self.lib.bfhe_mul_plain(self.h, _ptr(a), _ptr(plain), _ptr(out), n, self.stream))
        return out

    def add_const(self, a, c, out=None):
        out = torch.empty_like(a) if out is None else out
        self._same(self._n(a), out)
        _check(self.lib.bfhe_add_const(self.h, _ptr(a), c, _ptr(out), self._n(a), self.stream))
        return out

    def sub_const(self, a, c, out=None):
        out = torch.empty_like(a) if out is None else out
        self._same(self._n(a), out)
        _check(self.lib.bfhe_sub_const(self.h, _ptr(a), c, _ptr(out), self._n(a), self.stream))
        return out

    def const_sub(self, c, a, out=None):
        out = torch.empty_like(a) if out is None else out
        self._same(self._n(a), out)
        _check(self.lib.bfhe_const_sub(self.h, c, _ptr(a), _ptr(out), self._n(a), self.stream))
        return out

    def mul_scalar(self, a, c, out=None):
        out = torch.empty_like(a) if out is None else out
        self._same(self._n(a), out)
        _check(self.lib.bfhe_mul_scalar(self.h, _ptr(a), c, _ptr(out), self._n(a), self.stream))
        return out

    def bit_gate(self, gate, x, y=None, z=None, out=None):
        out = torch.empty_like(x) if out is None else out
        self._same(self._n(x), y, z, out)
        _check(self.lib.bfhe_bit_gate(self.h, gate, _ptr(x), _ptr(y), _ptr(z), _ptr(out), self._n(x),
                                      self.stream))
        return out

    def gate_level(self, wires, table, n_gates, n_mul):
        """wires [n_wires][n][2][L][N]; table: device int32 [n_gates][5], multiplying gates first."""
        n_wires, n = wires.shape[0], wires.shape[1]
        _check(self.lib.bfhe_gate_level(self.h, _ptr(wires), n_wires, n, _ptr(table), n_gates, n_mul,
                                        self.stream))

    def bits_to_mod(self, bits, out=None):
        s, n = bits.shape[0], bits.shape[1]
        self._same(s * n, bits)
        out = self.empty_ct(n) if out is None else out
        self._same(n, out)
        _check(self.lib.bfhe_bits_to_mod(self.h, _ptr(bits), s, _ptr(out), n, self.stream))
        return out

    def mod_to_bits(self, x, s, c_lo, c_hi, mode=PAPER, out=None):
        n = self._n(x)
        out = self.empty_ct(n, s) if out is None else out
        self._same(s * n, out)
        _check(self.lib.bfhe_mod_to_bits(self.h, _ptr(x), s, c_lo, c_hi, mode, _ptr(out), n, self.stream))
        return out

    def sint_to_mod(self, bits, out=None):
        """bits [s][n][2][L][N]: two's complement, sign bit last (Listing 6)."""
        s, n = bits.shape[0], bits.shape[1]
        self._same(s * n, bits)
        out = self.empty_ct(n) if out is None else out
        self._same(n, out)
        _check(self.lib.bfhe_sint_to_mod(self.h, _ptr(bits), s, _ptr(out), n, self.stream))
        return out

    def mod_to_sint(self, x, s, pos_range, neg_range, mode=PAPER, out=None):
        """Listing 9; pos_range / neg_range = (lo, hi) candidates of x and of (2^s - t) + x."""
        n = self._n(x)
        out = self.empty_ct(n, s) if out is None else out
        self._same(s * n, out)
        _check(self.lib.bfhe_mod_to_sint(self.h, _ptr(x), s, pos_range[0], pos_range[1], neg_range[0],
                                         neg_range[1], mode, _ptr(out), n, self.stream))
        return out

    def pow(self, x, e, out=None):
        out = torch.empty_like(x) if out is None else out
        self._same(self._n(x), out)
        _check(self.lib.bfhe_pow(self.h, _ptr(x), e, _ptr(out), self._n(x), self.stream))
        return out

    def op_counts(self, reset=False):
        buf = (ctypes.c_uint64 * 4)()
        _check(self.lib.bfhe_op_counts(self.h, buf, int(reset)))
        return tuple(int(v) for v in buf)

    def ntt(self, data, inverse=False):
        """In place over the first data.shape[-2] data primes: data [n_polys][n_limbs][N]."""
        n_limbs = data.shape[-2]
        n_polys = data.numel() // (n_limbs * self.N)
        _check(self.lib.bfhe_ntt(self.h, _ptr(data), n_polys, n_limbs, int(inverse), self.stream))
        return data

    def profile(self, enable):
        _check(self.lib.bfhe_profile(self.h, int(enable)))

    def profile_read(self):
        """{class: (ms, launches, modmuls, algorithmic DRAM bytes)} since the last read (synchronises)."""
        ms = (ctypes.c_double * len(KERNEL_CLASSES))()
        cnt = (ctypes.c_uint64 * len(KERNEL_CLASSES))()
        work = (ctypes.c_double * len(KERNEL_CLASSES))()
        nbytes = (ctypes.c_double * len(KERNEL_CLASSES))()
        _check(self.lib.bfhe_profile_read(self.h, ms, cnt, work, nbytes))
        return {k: (ms[i], int(cnt[i]), work[i], nbytes[i]) for i, k in enumerate(KERNEL_CLASSES)}


def probe_modmul(device=0, iters=1 << 14):
    """Measured 64-bit Shoup modmul rate of this GPU (modmul/s)."""
    lib = load()
    out = ctypes.c_double()
    _check(lib.bfhe_probe_modmul(device, iters, ctypes.byref(out),
                                 ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)))
    return out.value


def launch_count():
    """Kernels launched by the library so far in this process."""
    return int(load().bfhe_launch_count())


def ntt_config(logN, inverse, log_m=0, log_e=0):
    """Set (log_m != 0) and return the NTT block shape (log_m, log_e) for ring degree 2^logN."""
    m, e = ctypes.c_uint32(), ctypes.c_uint32()
    _check(load().bfhe_ntt_config(logN, int(inverse), log_m, log_e, ctypes.byref(m), ctypes.byref(e)))
    return m.value, e.value


def set_mul_tile(logN, max_ct):
    """Most ciphertexts per multiply launch sequence at ring degree 2^logN (0: as the scratch allows)."""
    _check(load().bfhe_set_mul_tile(logN, max_ct))


def mul_tile(logN):
    return int(load().bfhe_mul_tile(logN))


def set_scratch_budget(nbytes):
    """Per-call scratch budget in bytes (process-wide); larger batches are tiled."""
    _check(load().bfhe_set_scratch_budget(int(nbytes)))


def scratch_budget():
    return int(load().bfhe_scratch_budget())


def param_primes(N, L, alpha, t=65537, prime_bits=50):
    """Moduli (data, special, auxiliary) and K of the parameter rule, computed on the host."""
    lib = load()
    prm = _Params(N, L, alpha, prime_bits, t)
    buf = (ctypes.c_uint64 * 80)()
    K = ctypes.c_uint32(0)
    _check(lib.bfhe_param_primes(ctypes.byref(prm), buf, ctypes.byref(K)))
    return [int(buf[i]) for i in range(L + alpha + K.value)], K.value
