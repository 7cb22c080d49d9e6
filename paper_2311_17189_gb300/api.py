"""Python surface of libtami: a Diagram handle over the C ABI (include/tami.h).

Arrays on the device are torch tensors (complex128 / float64, CUDA); the calls run on
torch's current CUDA stream.  Host-only calls (construction, info, enumeration) take and
return numpy arrays.
"""
import contextlib
import ctypes
import os

import numpy as np

from . import _lib as L


def _torch():
    import torch
    return torch


def _nvtx(name):
    """An NVTX range around a library call when TAMI_NVTX=1 (for timeline profilers); else nothing."""
    if os.environ.get("TAMI_NVTX") == "1":
        return _torch().cuda.nvtx.range(name)
    return contextlib.nullcontext()


def _stream_ptr():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _as_c_pairs(X, device, n_ext=1):
    """complex [n_f] (or [n_f, n_ext]: one row of external frequencies per f) -> contiguous
    float64 [n_f, 2] ([n_f, n_ext, 2]) on `device`."""
    torch = _torch()
    X = torch.as_tensor(X)
    if not torch.is_complex(X):
        X = X.to(torch.complex128)
    X = X.to(device=device, dtype=torch.complex128).reshape(-1) if n_ext == 1 else \
        X.to(device=device, dtype=torch.complex128).reshape(-1, n_ext)
    return torch.view_as_real(X).contiguous()


JIT_MODES = {"never": L.TAMI_JIT_NEVER, "auto": L.TAMI_JIT_AUTO, "always": L.TAMI_JIT_ALWAYS}


def set_jit(mode):
    """Which kernel forward_backward runs (tami_set_jit): 'never' the generic kernel, 'auto' (the
    default) the diagram's specialised kernel for launches of >= 2^21 samples, 'always' the
    specialised kernel for every launch.  Process-wide."""
    L.check(L.lib().tami_set_jit(JIT_MODES[mode]))


STAGING_MODES = {"auto": L.TAMI_STAGING_AUTO, "streamed": L.TAMI_STAGING_STREAMED}


def set_table_staging(mode, chunk_ops=0):
    """How the generic forward kernels stage a table (tami_set_table_staging): 'auto' keeps the
    pole-DAG program resident in shared memory when it fits beside the tiles and streams it in
    chunks otherwise, 'streamed' always streams it (same bits); chunk_ops even in [16, 4096], 0
    keeps the current chunk size.  Process-wide."""
    L.check(L.lib().tami_set_table_staging(STAGING_MODES[mode], int(chunk_ops)))


def debug_set_wait_limit(first_stage_spins):
    """Test hook (tami_debug_set_wait_limit): bound the first stage of the generic kernels'
    mbarrier waits; -1 restores the default."""
    L.check(L.lib().tami_debug_set_wait_limit(int(first_stage_spins)))


class Diagram:
    """An AMI solution (flat terms A * FT * R, Sec. 2.2) and its device term table.  The last
    n_ext columns of alpha are external variables (Sec. 2.3); the others are summed.  Momentum
    sampling (forward, backward, batches) takes n_ext = 1; eval_energies any n_ext."""

    def __init__(self, alpha, eps=None, var_is_boson=None, order=None, prefactor=1.0, n_ext=1):
        a = np.ascontiguousarray(np.asarray(alpha, dtype=np.int8))
        self.alpha = a
        self.n_lines, self.n_vars = a.shape
        self.n_ext = int(n_ext)
        e = None if eps is None else np.ascontiguousarray(np.asarray(eps, dtype=np.int8))
        b = None if var_is_boson is None else np.ascontiguousarray(np.asarray(var_is_boson, dtype=np.uint8))
        o = None if order is None else np.ascontiguousarray(np.asarray(order, dtype=np.int32))
        h = ctypes.c_void_p()
        L.check(L.lib().tami_construct_ext(self.n_lines, self.n_vars, self.n_ext, L._np_ptr(a), L._np_ptr(e),
                                           L._np_ptr(b), L._np_ptr(o), float(prefactor), ctypes.byref(h)))
        self._h = h
        self.device = None
        self._ws = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                L.lib().tami_destroy(h)
            except Exception:
                pass
            self._h = None

    def info(self):
        i = L.Info()
        L.check(L.lib().tami_diagram_info(self._h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in L.Info._fields_}

    def _dev(self):
        if self.device is None:
            raise L.TamiError(L.TAMI_EINVAL, "diagram not uploaded (call upload)")
        return f"cuda:{self.device}"

    def jit_prepare(self):
        """Build the specialised kernels of this uploaded diagram now (tami_jit_prepare)."""
        torch = _torch()
        with torch.cuda.device(self.device):
            L.check(L.lib().tami_jit_prepare(self._h))

    JIT_KINDS = {"fused": 0, "forward": 1, "adjoint": 2, "energy": 3}

    def jit_status(self):
        """Specialised kernels (tami_jit_status, tami_jit_cached): ready = set of built kinds
        ('fused', 'forward', 'adjoint', 'energy'), last_used = whether the last evaluating call ran
        one, compile_ms, cached = the built kinds loaded from the disk cache."""
        r, u, ms, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
        L.check(L.lib().tami_jit_status(self._h, ctypes.byref(r), ctypes.byref(u), ctypes.byref(ms)))
        L.check(L.lib().tami_jit_cached(self._h, ctypes.byref(c)))
        ready = {k for k, b in self.JIT_KINDS.items() if r.value & (1 << b)}
        cached = {k for k, b in self.JIT_KINDS.items() if c.value & (1 << b)}
        return {"ready": ready, "last_used": bool(u.value), "compile_ms": ms.value, "cached": cached}

    def jit_source(self, kind="fused"):
        """The CUDA C++ source of one specialised kernel (tami_jit_source)."""
        k = self.JIT_KINDS[kind]
        n = ctypes.c_size_t()
        L.check(L.lib().tami_jit_source(self._h, k, None, 0, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        L.check(L.lib().tami_jit_source(self._h, k, buf, n.value, ctypes.byref(n)))
        return buf.value.decode()

    def upload(self, device=None):
        torch = _torch()
        dev = torch.cuda.current_device() if device is None else int(device)
        with torch.cuda.device(dev):
            L.check(L.lib().tami_upload(self._h, dev, _stream_ptr()))
        self.device = dev
        return self

    # ---------------------------------------------------------------- evaluation
    def sample_energies(self, lattice, seed, offset, n):
        torch = _torch()
        E = torch.empty((n, self.n_lines), dtype=torch.float64, device=self._dev())
        lat = L.Lattice(*[float(v) for v in lattice])
        L.check(L.lib().tami_sample_energies(self._h, ctypes.byref(lat), int(seed), int(offset), int(n),
                                             ctypes.c_void_p(E.data_ptr()), _stream_ptr()))
        return E

    def eval_energies(self, E, X, beta):
        """E: float64 [n_e, n_lines] CUDA tensor; X: complex [n_f] (n_ext = 1) or [n_f, n_ext] (row f:
        the external frequencies in label order).  Returns complex128 [n_f, n_e]."""
        torch = _torch()
        E = E.to(dtype=torch.float64).contiguous()
        Xp = _as_c_pairs(X, E.device, self.n_ext)
        n_e, n_f = E.shape[0], Xp.shape[0]
        out = torch.empty((n_f, n_e, 2), dtype=torch.float64, device=E.device)
        with _nvtx("tami_eval_energies"):
            L.check(L.lib().tami_eval_energies(self._h, ctypes.c_void_p(E.data_ptr()), n_e,
                                               ctypes.c_void_p(Xp.data_ptr()), n_f, float(beta),
                                               ctypes.c_void_p(out.data_ptr()), _stream_ptr()))
        return torch.view_as_complex(out)

    def workspace(self, n, n_f):
        torch = _torch()
        nbytes = ctypes.c_size_t()
        L.check(L.lib().tami_forward_workspace(self._h, int(n), int(n_f), ctypes.byref(nbytes)))
        need = (nbytes.value + 255) // 256 * 256
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device=self._dev())
        return self._ws

    def saved_buffer(self, n):
        """A buffer for forward(save=...) / backward(saved=...): float64 [saved_rows, n]."""
        torch = _torch()
        return torch.empty((self.info()["saved_rows"], int(n)), dtype=torch.float64, device=self._dev())

    def forward(self, lattice, seed, offset, n, X, beta, per_sample=False, out=None, save=None):
        """Monte Carlo mean over n momentum samples (Sec. 5.2).  Returns (mean complex [n_f],
        var float64 [n_f, 2], per-sample complex [n_f, n] or None).  With save (a tensor from
        saved_buffer(n)) the per-sample line energies and dE/dK factors are written there for a
        backward() over the same samples."""
        torch = _torch()
        dev = self._dev()
        Xp = _as_c_pairs(X, dev)
        n_f = Xp.shape[0]
        if out is None:
            mean = torch.empty((n_f, 2), dtype=torch.float64, device=dev)
            var = torch.empty((n_f, 2), dtype=torch.float64, device=dev)
        else:
            mean, var = out
        ps = torch.empty((n_f, n, 2), dtype=torch.float64, device=dev) if per_sample else None
        if save is not None and (save.dtype != torch.float64 or not save.is_contiguous() or
                                 tuple(save.shape) != (self.info()["saved_rows"], int(n))):
            raise L.TamiError(L.TAMI_EINVAL, "save must be a contiguous float64 [saved_rows, n] tensor")
        ws = self.workspace(n, n_f)
        lat = L.Lattice(*[float(v) for v in lattice])
        with _nvtx("tami_forward"):
            L.check(L.lib().tami_forward(self._h, ctypes.byref(lat), int(seed), int(offset), int(n),
                                         ctypes.c_void_p(Xp.data_ptr()), n_f, float(beta),
                                         ctypes.c_void_p(mean.data_ptr()), ctypes.c_void_p(var.data_ptr()),
                                         ctypes.c_void_p(ps.data_ptr()) if ps is not None else None,
                                         ctypes.c_void_p(save.data_ptr()) if save is not None else None,
                                         ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr()))
        return (torch.view_as_complex(mean), var, torch.view_as_complex(ps) if ps is not None else None)

    def backward(self, lattice, seed, offset, n, X, beta, gout, per_sample=False, saved=None):
        """Adjoint of forward()'s mean for the upstream gradient gout (complex [n_f]).
        Returns dict: dSigma_dX (complex [n_f]), grad_X_re (float64 [n_f]), grad_params
        (float64 [3]: mu, kx_ext, ky_ext) and, with per_sample, dX (complex [n_f, n]) and
        grads (float64 [n, 3]).  saved: the buffer a forward(save=...) over the same samples
        filled (then the energies are read, not recomputed; same results)."""
        torch = _torch()
        dev = self._dev()
        Xp = _as_c_pairs(X, dev)
        Gp = _as_c_pairs(gout, dev)
        n_f = Xp.shape[0]
        dX = torch.empty((n_f, 2), dtype=torch.float64, device=dev)
        gX = torch.empty((n_f,), dtype=torch.float64, device=dev)
        gp = torch.empty((3,), dtype=torch.float64, device=dev)
        ps_dX = torch.empty((n_f, n, 2), dtype=torch.float64, device=dev) if per_sample else None
        ps_g = torch.empty((n, 3), dtype=torch.float64, device=dev) if per_sample else None
        if saved is not None and (saved.dtype != torch.float64 or not saved.is_contiguous() or
                                  tuple(saved.shape) != (self.info()["saved_rows"], int(n))):
            raise L.TamiError(L.TAMI_EINVAL, "saved must be a contiguous float64 [saved_rows, n] tensor")
        nbytes = ctypes.c_size_t()
        L.check(L.lib().tami_backward_workspace(self._h, int(n), n_f, ctypes.byref(nbytes)))
        need = (nbytes.value + 255) // 256 * 256
        if getattr(self, "_bws", None) is None or self._bws.numel() < need:
            self._bws = torch.empty(need, dtype=torch.uint8, device=dev)
        ws = self._bws
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        lat = L.Lattice(*[float(v) for v in lattice])
        with _nvtx("tami_backward"):
            L.check(L.lib().tami_backward(self._h, ctypes.byref(lat), int(seed), int(offset), int(n), ptr(Xp), n_f,
                                          float(beta), ptr(Gp), ptr(dX), ptr(gX), ptr(gp), ptr(ps_dX), ptr(ps_g),
                                          ptr(saved), ptr(ws), ws.numel(), _stream_ptr()))
        out = {"dSigma_dX": torch.view_as_complex(dX), "grad_X_re": gX, "grad_params": gp}
        if per_sample:
            out["dX"] = torch.view_as_complex(ps_dX)
            out["grads"] = ps_g
        return out

    def forward_backward(self, lattice, seed, offset, n, X, beta, gout, per_sample=False):
        """forward() and backward() in one pass (tami_forward_backward), for an upstream gradient
        known beforehand.  Returns the union of their results: mean, var, dSigma_dX, grad_X_re,
        grad_params and, with per_sample, values (complex [n_f, n]), dX and grads."""
        torch = _torch()
        dev = self._dev()
        Xp = _as_c_pairs(X, dev)
        Gp = _as_c_pairs(gout, dev)
        n_f = Xp.shape[0]
        f64 = dict(dtype=torch.float64, device=dev)
        mean, var, dX = torch.empty((n_f, 2), **f64), torch.empty((n_f, 2), **f64), torch.empty((n_f, 2), **f64)
        gX, gp = torch.empty((n_f,), **f64), torch.empty((3,), **f64)
        ps = torch.empty((n_f, n, 2), **f64) if per_sample else None
        ps_dX = torch.empty((n_f, n, 2), **f64) if per_sample else None
        ps_g = torch.empty((n, 3), **f64) if per_sample else None
        nbytes = ctypes.c_size_t()
        L.check(L.lib().tami_forward_backward_workspace(self._h, int(n), n_f, ctypes.byref(nbytes)))
        need = (nbytes.value + 255) // 256 * 256
        if getattr(self, "_fws", None) is None or self._fws.numel() < need:
            self._fws = torch.empty(need, dtype=torch.uint8, device=dev)
        ws = self._fws
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        lat = L.Lattice(*[float(v) for v in lattice])
        with _nvtx("tami_forward_backward"):
            L.check(L.lib().tami_forward_backward(self._h, ctypes.byref(lat), int(seed), int(offset), int(n), ptr(Xp),
                                                  n_f, float(beta), ptr(Gp), ptr(mean), ptr(var), ptr(ps), ptr(dX),
                                                  ptr(gX), ptr(gp), ptr(ps_dX), ptr(ps_g), ptr(ws), ws.numel(),
                                                  _stream_ptr()))
        out = {"mean": torch.view_as_complex(mean), "var": var, "dSigma_dX": torch.view_as_complex(dX),
               "grad_X_re": gX, "grad_params": gp}
        if per_sample:
            out["values"] = torch.view_as_complex(ps)
            out["dX"] = torch.view_as_complex(ps_dX)
            out["grads"] = ps_g
        return out


class Batch:
    """Many diagrams in one persistent, graph-captured launch (tami_batch_*).  Each diagram d gets
    samples[d] Philox samples with key seeds[d]; the lattice and frequencies are shared.  Diagrams
    the specialised-kernel mode selects (set_jit) run their own generated forward kernel inside
    the same graph instead of the persistent kernel's work queue."""

    def __init__(self, diagrams, samples, seeds, n_f, chunk_tiles=0):
        torch = _torch()
        self.diagrams = list(diagrams)
        n_d = len(self.diagrams)
        hs = (ctypes.c_void_p * n_d)(*[d._h.value for d in self.diagrams])
        smp = np.ascontiguousarray(np.asarray(samples, dtype=np.int64))
        sd = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
        h = ctypes.c_void_p()
        L.check(L.lib().tami_batch_plan(ctypes.cast(hs, ctypes.c_void_p), n_d, L._np_ptr(smp), L._np_ptr(sd),
                                        int(n_f), int(chunk_tiles), ctypes.byref(h)))
        self._h = h
        self.n_d, self.n_f = n_d, int(n_f)
        self.device = torch.cuda.current_device()

    def info(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        L.check(L.lib().tami_batch_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        flags = (ctypes.c_int * self.n_d)()
        n_spec = ctypes.c_int()
        L.check(L.lib().tami_batch_specialised(self._h, flags, ctypes.byref(n_spec)))
        return {"items": a.value, "grid": b.value, "chunk_tiles": c.value, "specialised": n_spec.value,
                "specialised_diagrams": [d for d in range(self.n_d) if flags[d]]}

    def debug_set_item(self, item, d, tile0, tile1):
        """Overwrite one entry of the device work queue (tami_batch_debug_set_item); returns the
        previous entry (d, tile0, tile1)."""
        prev = (ctypes.c_int64 * 3)()
        L.check(L.lib().tami_batch_debug_set_item(self._h, int(item), int(d), int(tile0), int(tile1), prev))
        return tuple(int(v) for v in prev)

    def launch(self, lattice, X, beta, out=None):
        """Returns (mean complex [n_d, n_f], var float64 [n_d, n_f, 2])."""
        torch = _torch()
        dev = f"cuda:{self.device}"
        Xp = _as_c_pairs(X, dev)
        if out is None:
            mean = torch.empty((self.n_d, self.n_f, 2), dtype=torch.float64, device=dev)
            var = torch.empty((self.n_d, self.n_f, 2), dtype=torch.float64, device=dev)
        else:
            mean, var = out
        lat = L.Lattice(*[float(v) for v in lattice])
        with _nvtx("tami_batch_launch"):
            L.check(L.lib().tami_batch_launch(self._h, ctypes.byref(lat), ctypes.c_void_p(Xp.data_ptr()), float(beta),
                                              ctypes.c_void_p(mean.data_ptr()), ctypes.c_void_p(var.data_ptr()),
                                              _stream_ptr()))
        return torch.view_as_complex(mean), var

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                L.lib().tami_batch_destroy(h)
            except Exception:
                pass
            self._h = None


def enumerate_sigma(order):
    """Hubbard self-energy diagrams of `order` (libtami's enumerator and labeller, Sec. 2.5):
    list of dicts with alpha [N, m+1], eps [N, N], code, loops, in canonical order."""
    m = int(order)
    N, nv = 2 * m - 1, m + 1
    n = ctypes.c_int()
    L.check(L.lib().tami_enumerate_sigma(m, 0, None, None, None, None, ctypes.byref(n)))
    cnt = n.value
    a = np.zeros((cnt, N, nv), dtype=np.int8)
    e = np.zeros((cnt, N, N), dtype=np.int8)
    c = np.zeros((cnt, 2 * m + 1), dtype=np.int32)
    lo = np.zeros(cnt, dtype=np.int32)
    L.check(L.lib().tami_enumerate_sigma(m, cnt, L._np_ptr(a), L._np_ptr(e), L._np_ptr(c), L._np_ptr(lo),
                                         ctypes.byref(n)))
    return [{"alpha": a[i], "eps": e[i], "code": tuple(int(v) for v in c[i]), "loops": int(lo[i])}
            for i in range(cnt)]


def construct_many(specs, threads=None):
    """Diagrams for many label sets at once: each spec is a dict of Diagram's arguments (alpha,
    and optionally eps, var_is_boson, order, prefactor, n_ext).  The constructions run on a pool of
    host threads (libtami's construction keeps no shared state, and the ctypes call releases the
    interpreter lock); the result is in the order of `specs`, the first failure is raised."""
    from concurrent.futures import ThreadPoolExecutor
    specs = list(specs)
    if not specs:
        return []
    workers = max(1, min(len(specs), int(threads) if threads else (os.cpu_count() or 1)))
    if workers == 1:
        return [Diagram(**sp) for sp in specs]
    with ThreadPoolExecutor(max_workers=workers) as pool:
        return list(pool.map(lambda sp: Diagram(**sp), specs))
