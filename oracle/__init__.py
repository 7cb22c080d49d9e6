"""CPU oracle for algorithmic Matsubara integration -- TEST INFRASTRUCTURE ONLY.

A plain, slow FP64 restatement of the method of arXiv:2311.17189 (construction by repeated
(multipole) residues, Sec. 2.2; term-by-term evaluation, Sec. 2.3; momentum sampling,
Sec. 5.2), written in C++ (ami_oracle.cpp) and loaded here with ctypes.  Only tests/,
__graft_entry__.smoke() and bench.py's CPU-baseline leg may import this package; the library
in paper_2311_17189_gb300/ never does, and the two share no code.

Parity status of each function (what pins it) is stated in tests/test_oracle_*.py.  The
enumerator's diagram set is cross-checked against the library's own enumerator and pinned by the
half-filled Hubbard atom (tests/test_oracle_atomic.py): its exact self-energy U/2 + U^2/(4 i omega)
fixes every order's sum, which the enumerated diagrams reach as the line energies go to zero (down
to a single diagram at orders 2-4; at order 5 only diagrams above a few per cent of the largest).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        i32p, dp, u32p = P(ctypes.c_int), P(ctypes.c_double), P(ctypes.c_uint32)
        i64p = P(ctypes.c_int64)
        L.orc_last_error.restype = ctypes.c_char_p
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_sincos.argtypes = [dp, ctypes.c_int64, dp, dp]
        L.orc_fermi_deriv.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.orc_fermi_deriv.restype = ctypes.c_double
        L.orc_construct.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, i32p, i32p, ctypes.c_double]
        L.orc_construct.restype = ctypes.c_void_p
        L.orc_construct_ext.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i32p, i32p, i32p, i32p,
                                        ctypes.c_double]
        L.orc_construct_ext.restype = ctypes.c_void_p
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_info.argtypes = [ctypes.c_void_p, i64p]
        L.orc_term.argtypes = [ctypes.c_void_p, ctypes.c_int64, dp, i32p, i32p, i32p, i32p, i32p, i32p,
                               i32p, ctypes.c_int]
        L.orc_eval_energies.argtypes = [ctypes.c_void_p, dp, ctypes.c_int64, dp, dp, ctypes.c_int,
                                        ctypes.c_double, dp, dp, dp, dp, dp, ctypes.c_int]
        L.orc_sample_energies.argtypes = [ctypes.c_int, ctypes.c_int, i32p, dp, ctypes.c_uint64,
                                          ctypes.c_uint64, ctypes.c_int64, dp, dp]
        L.orc_eval_momenta.argtypes = [ctypes.c_void_p, i32p, dp, ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.c_int64, dp, dp, ctypes.c_int, ctypes.c_double, dp, dp, dp,
                                       dp, dp, dp, ctypes.c_int]
        L.orc_eval_momenta_deriv.argtypes = [ctypes.c_void_p, i32p, dp, ctypes.c_uint64, ctypes.c_uint64,
                                             ctypes.c_int64, dp, dp, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_int, dp, dp, dp, dp, dp, dp, dp, ctypes.c_int]
        L.orc_eval_energies_deriv.argtypes = [ctypes.c_void_p, dp, dp, ctypes.c_int64, dp, dp, dp, dp,
                                              ctypes.c_int, ctypes.c_double, dp, dp, dp]
        L.orc_eval_momenta.restype = ctypes.c_int
        L.orc_eval_momenta_deriv.restype = ctypes.c_int
        L.orc_brute_force.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i32p, i32p, i32p, dp, dp, dp,
                                      ctypes.c_double, ctypes.c_int, dp]
        L.orc_enumerate_sigma.argtypes = [ctypes.c_int]
        L.orc_diagram.argtypes = [ctypes.c_int, i32p, i32p, i32p, dp, i32p]
        _lib = L
    return _lib


def _ptr(a, ct):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _i32(a):
    return None if a is None else np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _f64(a):
    return None if a is None else np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _err():
    return lib().orc_last_error().decode()


def _chk(rc):
    if rc != 0:
        raise ValueError("oracle: " + _err())


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out


def sincos(k):
    k = _f64(k).ravel()
    s = np.empty_like(k)
    c = np.empty_like(k)
    lib().orc_sincos(_ptr(k, ctypes.c_double), k.size, _ptr(s, ctypes.c_double), _ptr(c, ctypes.c_double))
    return s, c


def fermi_deriv(sigma, k, beta, x):
    return lib().orc_fermi_deriv(int(sigma), int(k), float(beta), float(x))


def _rows(X, n_ext):
    """External frequencies as contiguous (re, im) arrays [n_f, n_ext]: X is [n_f] (n_ext = 1) or
    [n_f, n_ext]."""
    X = np.asarray(X, dtype=np.complex128).reshape(-1, n_ext)
    return _f64(X.real), _f64(X.imag), X.shape[0]


class Solution:
    """AMI solution built by the oracle (flat terms).  The last n_ext columns of alpha are the
    external variables (Sec. 2.3); the others are summed."""

    def __init__(self, alpha, eps=None, var_is_boson=None, order=None, prefactor=1.0, n_ext=1):
        alpha = _i32(alpha)
        self.alpha = alpha
        self.N, self.nv = alpha.shape
        self.n_ext = int(n_ext)
        self.eps = _i32(eps)
        self.boson = _i32(var_is_boson)
        self.order = _i32(order)
        h = lib().orc_construct_ext(self.N, self.nv, self.n_ext, _ptr(alpha, ctypes.c_int),
                                    _ptr(self.eps, ctypes.c_int), _ptr(self.boson, ctypes.c_int),
                                    _ptr(self.order, ctypes.c_int), float(prefactor))
        if not h:
            raise ValueError("oracle construct failed: " + _err())
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def info(self):
        out = np.zeros(7, dtype=np.int64)
        lib().orc_info(self._h, _ptr(out, ctypes.c_int64))
        keys = ["terms", "fermi_factors", "g_factors", "max_der", "max_g", "unique_poles", "unique_dens"]
        return dict(zip(keys, (int(v) for v in out)))

    def term(self, t, cap=64):
        A = ctypes.c_double()
        nF, nG = ctypes.c_int(), ctypes.c_int()
        fc = np.zeros(cap * self.N, dtype=np.int32)
        fs = np.zeros(cap, dtype=np.int32)
        fk = np.zeros(cap, dtype=np.int32)
        ge = np.zeros(cap * self.N, dtype=np.int32)
        ga = np.zeros(cap * self.n_ext, dtype=np.int32)
        rc = lib().orc_term(self._h, int(t), ctypes.byref(A), ctypes.byref(nF), _ptr(fc, ctypes.c_int),
                            _ptr(fs, ctypes.c_int), _ptr(fk, ctypes.c_int), ctypes.byref(nG),
                            _ptr(ge, ctypes.c_int), _ptr(ga, ctypes.c_int), cap)
        if rc != 0:
            raise ValueError(_err())
        F = [(tuple(fc[i * self.N:(i + 1) * self.N]), int(fs[i]), int(fk[i])) for i in range(nF.value)]
        if self.n_ext == 1:
            G = [(tuple(ge[i * self.N:(i + 1) * self.N]), int(ga[i])) for i in range(nG.value)]
        else:
            G = [(tuple(ge[i * self.N:(i + 1) * self.N]), tuple(ga[i * self.n_ext:(i + 1) * self.n_ext]))
                 for i in range(nG.value)]
        return A.value, F, G

    def eval_energies(self, E, X, beta, threads=1, sens=False):
        """E: [n_e, N] base energies; X: [n_f] complex (n_ext = 1) or [n_f, n_ext] (one row of
        external frequencies per f).  Returns (values [n_f, n_e] complex, sum|term| [n_f, n_e],
        envelope [n_f, n_e]) and, with sens=True, the energy sensitivity
        sum_t sum_j |d term_t / d E_j| [n_f, n_e] as a fourth item."""
        E = _f64(E)
        n_e = E.shape[0]
        xr, xi, nf = _rows(X, self.n_ext)
        vr = np.empty((nf, n_e)); vi = np.empty((nf, n_e))
        ab = np.empty((nf, n_e)); en = np.empty((nf, n_e))
        sn = np.empty((nf, n_e)) if sens else None
        d = ctypes.c_double
        lib().orc_eval_energies(self._h, _ptr(E, d), n_e, _ptr(xr, d), _ptr(xi, d), nf, float(beta),
                                _ptr(vr, d), _ptr(vi, d), _ptr(ab, d), _ptr(en, d), _ptr(sn, d), int(threads))
        if sens:
            return vr + 1j * vi, ab, en, sn
        return vr + 1j * vi, ab, en

    def eval_momenta(self, lattice, seed, offset, n, X, beta, per_sample=True, threads=1, alpha=None):
        """Momentum-sampled evaluation.  lattice = (t, t', mu, kx_ext, ky_ext).  Returns dict with
        mean [n_f] complex, var [n_f, 2], and (if per_sample) values, envelope (the rounding
        envelope) and sens (sum_t sum_j |d term_t / d E_j|, the first-order change per unit change
        of every base energy) [n_f, n]."""
        a = self.alpha if alpha is None else _i32(alpha)
        lat = _f64(lattice)
        X = np.asarray(X, dtype=np.complex128).ravel()
        xr, xi = _f64(X.real), _f64(X.imag)
        nf = X.size
        d = ctypes.c_double
        mean = np.empty(2 * nf); var = np.empty(2 * nf)
        vr = vi = en = sn = None
        if per_sample:
            vr = np.empty((nf, n)); vi = np.empty((nf, n)); en = np.empty((nf, n)); sn = np.empty((nf, n))
        _chk(lib().orc_eval_momenta(self._h, _ptr(a, ctypes.c_int), _ptr(lat, d), int(seed), int(offset), int(n),
                               _ptr(xr, d), _ptr(xi, d), nf, float(beta), _ptr(vr, d), _ptr(vi, d),
                               _ptr(en, d), _ptr(sn, d), _ptr(mean, d), _ptr(var, d), int(threads)))
        out = {"mean": mean[0::2] + 1j * mean[1::2], "var": var.reshape(nf, 2)}
        if per_sample:
            out["values"] = vr + 1j * vi
            out["envelope"] = en
            out["sens"] = sn
        return out

    def eval_momenta_deriv(self, lattice, seed, offset, n, X, beta, which, threads=1, alpha=None,
                           envelope=False, sens=False):
        """Per-sample dual-number derivative [n_f, n] along which in
        {'omega', 'mu', 'kx', 'ky'}; returns (values, derivatives), with envelope=True
        (values, derivatives, derivative rounding envelope), and with sens=True also the energy
        sensitivities of the derivative and of the value (sum_t sum_j |d (d term_t) / d E_j| and
        sum_t sum_j |d term_t / d E_j|), in that order."""
        w = {"omega": 0, "mu": 1, "kx": 2, "ky": 3}[which]
        a = self.alpha if alpha is None else _i32(alpha)
        lat = _f64(lattice)
        X = np.asarray(X, dtype=np.complex128).ravel()
        xr, xi = _f64(X.real), _f64(X.imag)
        nf = X.size
        d = ctypes.c_double
        vr = np.empty((nf, n)); vi = np.empty((nf, n)); dr = np.empty((nf, n)); di = np.empty((nf, n))
        de = np.empty((nf, n))
        sv = ds = None
        if sens:
            sv = np.empty((nf, n)); ds = np.empty((nf, n))
        _chk(lib().orc_eval_momenta_deriv(self._h, _ptr(a, ctypes.c_int), _ptr(lat, d), int(seed), int(offset),
                                          int(n), _ptr(xr, d), _ptr(xi, d), nf, float(beta), w, _ptr(vr, d),
                                          _ptr(vi, d), _ptr(dr, d), _ptr(di, d), _ptr(de, d), _ptr(sv, d),
                                          _ptr(ds, d), int(threads)))
        if sens:
            return vr + 1j * vi, dr + 1j * di, de, ds, sv
        if envelope:
            return vr + 1j * vi, dr + 1j * di, de
        return vr + 1j * vi, dr + 1j * di

    def eval_energies_deriv(self, E, dE, X, dX, beta, sens=False):
        """Dual-number derivative [n_f, n_e] along dE (base energies, [n_e, N]) and dX (the
        external frequencies' direction, scalar or [n_ext], the same for every row of X); with
        sens=True also the derivative's energy sensitivity sum_t sum_j |d (d term_t) / d E_j|."""
        E = _f64(E); dE = _f64(dE)
        n_e = E.shape[0]
        xr, xi, nf = _rows(X, self.n_ext)
        dXv = np.broadcast_to(np.asarray(dX, dtype=np.complex128).ravel(), (self.n_ext,))
        dxr, dxi = _f64(dXv.real), _f64(dXv.imag)
        d = ctypes.c_double
        dr = np.empty((nf, n_e)); di = np.empty((nf, n_e))
        ds = np.empty((nf, n_e)) if sens else None
        lib().orc_eval_energies_deriv(self._h, _ptr(E, d), _ptr(dE, d), n_e, _ptr(xr, d), _ptr(xi, d),
                                      _ptr(dxr, d), _ptr(dxi, d), nf, float(beta), _ptr(dr, d), _ptr(di, d),
                                      _ptr(ds, d))
        if sens:
            return dr + 1j * di, ds
        return dr + 1j * di


def sample_energies(alpha, lattice, seed, offset, n):
    a = _i32(alpha)
    N, nv = a.shape
    m = nv - 1
    lat = _f64(lattice)
    E = np.empty((n, N)); k = np.empty((n, m, 2))
    d = ctypes.c_double
    lib().orc_sample_energies(N, nv, _ptr(a, ctypes.c_int), _ptr(lat, d), int(seed), int(offset), int(n),
                              _ptr(E, d), _ptr(k, d))
    return E, k


def brute_force(alpha, E, X, beta, nmax, eps=None, var_is_boson=None, n_ext=1):
    """Truncated Matsubara sum of prod_j G_j over the first nv - n_ext variables; X: the n_ext
    external frequencies (scalar for n_ext = 1)."""
    a = _i32(alpha)
    N, nv = a.shape
    E = _f64(E)
    xr, xi, _ = _rows(X, n_ext)
    out = np.empty(2)
    d = ctypes.c_double
    _chk(lib().orc_brute_force(N, nv, int(n_ext), _ptr(a, ctypes.c_int), _ptr(_i32(eps), ctypes.c_int),
                               _ptr(_i32(var_is_boson), ctypes.c_int), _ptr(E, d), _ptr(xr, d), _ptr(xi, d),
                               float(beta), int(nmax), _ptr(out, d)))
    return out[0] + 1j * out[1]


def enumerate_sigma(order):
    """Hubbard self-energy diagrams of the given order: list of dicts with alpha, eps, code,
    sign (-1)^F and loops F, in canonical-code order."""
    n = lib().orc_enumerate_sigma(int(order))
    if n < 0:
        raise ValueError(_err())
    m = order
    N = 2 * m - 1
    out = []
    for i in range(n):
        a = np.zeros(N * (m + 1), dtype=np.int32)
        e = np.zeros(N * N, dtype=np.int32)
        c = np.zeros(1 + 2 * m, dtype=np.int32)
        s = ctypes.c_double()
        lo = ctypes.c_int()
        lib().orc_diagram(i, _ptr(a, ctypes.c_int), _ptr(e, ctypes.c_int), _ptr(c, ctypes.c_int),
                          ctypes.byref(s), ctypes.byref(lo))
        out.append({"alpha": a.reshape(N, m + 1), "eps": e.reshape(N, N), "code": tuple(int(v) for v in c),
                    "sign": s.value, "loops": lo.value})
    return out
