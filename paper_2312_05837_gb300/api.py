"""Python binding of the C ABI (include/ising_ds.h): argument marshalling only.

Every function takes an instance object with the attributes ``n, layout, J,
indptr, indices, data, h, j_scale, convention`` (numpy arrays for host memory,
or torch CUDA tensors for device memory) and calls the matching ``ising_*``
entry point. Nothing here computes any part of the method.
"""

from __future__ import annotations

import ctypes
import weakref
from ctypes import byref, c_double, c_int32, c_int64, c_void_p

import numpy as np

from . import _lib as L

_NP_DT = {np.dtype(np.float64): L.F64, np.dtype(np.float32): L.F32,
          np.dtype(np.int8): L.I8, np.dtype(np.int32): L.I32}
_PREC = {"auto": L.PREC_AUTO, "fp32": L.PREC_FP32_PLAIN, "plain": L.PREC_FP32_PLAIN,
         "tc": L.PREC_TC, "bf16": L.PREC_BF16, "fp8": L.PREC_FP8}


class IsingError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"ising error {code}: {msg}")
        self.code = code


def _torch():
    import torch
    return torch


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _is_dev(x) -> bool:
    return _is_torch(x) and x.is_cuda


def _dtype_code(x) -> int:
    if _is_torch(x):
        t = _torch()
        m = {t.float64: L.F64, t.float32: L.F32, t.int8: L.I8, t.int32: L.I32}
        return m[x.dtype]
    return _NP_DT[np.dtype(x.dtype)]


def _ptr(x) -> int:
    if x is None:
        return 0
    if _is_torch(x):
        assert x.is_contiguous()
        return x.data_ptr()
    assert x.flags["C_CONTIGUOUS"]
    return x.ctypes.data


def _host(x, dtype=None):
    if x is None:
        return None
    a = np.ascontiguousarray(x if dtype is None else np.asarray(x, dtype=dtype))
    return a


class Context:
    """A library context on one CUDA device and stream (default: torch's
    current stream on that device)."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = L.load()
        torch = _torch()
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self.device = device
        self.handle = c_void_p()
        self._children = weakref.WeakSet()  # sessions / pruning results using this context
        rc = self.lib.ising_create(byref(self.handle), device, c_void_p(stream))
        if rc != L.OK:
            raise IsingError(rc, "ising_create failed (no CUDA device?)")

    def check(self, rc: int):
        if rc != L.OK:
            msg = self.lib.ising_last_error(self.handle)
            raise IsingError(rc, msg.decode() if msg else "")

    def synchronize(self):
        self.check(self.lib.ising_synchronize(self.handle))

    def close(self):
        """Releases the context after every session / pruning result made on
        it (the library requires those to go first)."""
        if self.handle:
            # packs borrow sessions: close them first
            for child in sorted(self._children, key=lambda c: not isinstance(c, Pack)):
                child.close()
            self.lib.ising_destroy(self.handle)
            self.handle = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _conv(c) -> int:
    return L.CONV_PAPER if c in ("paper", L.CONV_PAPER) else L.CONV_PHYSICS


def make_instance(inst):
    """ctypes ising_instance for `inst` plus the arrays it points into."""
    keep = []
    dense = inst.layout == "dense"
    if dense:
        J = inst.J
    else:
        J = inst.data
    dev = _is_dev(J)
    if not dev:
        J = _host(J)
    keep.append(J)
    s = L.Instance()
    s.n = int(inst.n)
    s.layout = L.LAYOUT_DENSE if dense else L.LAYOUT_CSR
    s.j_dtype = _dtype_code(J)
    s.J = _ptr(J)
    if not dense:
        ip, ix = inst.indptr, inst.indices
        if not dev:
            ip = _host(ip, np.int64)
            ix = _host(ix, np.int32)
        keep += [ip, ix]
        s.indptr = _ptr(ip)
        s.indices = _ptr(ix)
        s.nnz = int(ip[-1])
    h = inst.h
    if h is not None:
        if not dev:
            h = _host(h)
            if h.dtype not in (np.float64, np.float32, np.int32):
                h = h.astype(np.float64)
        keep.append(h)
        s.h_dtype = _dtype_code(h)
        s.h = _ptr(h)
    s.j_scale = float(inst.j_scale)
    s.convention = _conv(inst.convention)
    s.mem = L.MEM_DEVICE if dev else L.MEM_HOST
    return s, keep


def params(restarts, steps, lr=6.0, mu=0.0, beta1=0.9, beta2=0.999, eps=1e-8, seed=0,
           precision="auto", profile=False, streaming=False, autotune=True,
           converge=False, relaxed=False) -> L.DSParams:
    p = L.DSParams()
    p.restarts = int(restarts)
    p.steps = int(steps)
    p.lr, p.mu, p.beta1, p.beta2, p.eps = float(lr), float(mu), float(beta1), float(beta2), float(eps)
    p.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    p.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
    p.flags = ((L.DS_PROFILE if profile else 0) | (L.DS_STREAMING if streaming else 0) |
               (0 if autotune else L.DS_NO_AUTOTUNE) | (L.DS_CONVERGE if converge else 0) |
               (L.DS_RELAXED if relaxed else 0))
    return p


def _stats_dict(st: L.DSStats) -> dict:
    return {f: getattr(st, f) for f, _ in L.DSStats._fields_}


def energy(ctx: Context, inst, spins, exact_parts: bool = False):
    """E(s) for spins[count][n] (int8); returns float64 energies (and the
    exact integer parts Q, H when asked)."""
    s, keep = make_instance(inst)
    dev = s.mem == L.MEM_DEVICE
    if dev:
        torch = _torch()
        sp = spins.to(torch.int8).contiguous()
        count = sp.shape[0] if sp.dim() == 2 else 1
        E = torch.empty(count, dtype=torch.float64, device=sp.device)
        Q = torch.empty(count, dtype=torch.int64, device=sp.device) if exact_parts else None
        H = torch.empty(count, dtype=torch.int64, device=sp.device) if exact_parts else None
    else:
        sp = _host(spins, np.int8)
        count = sp.shape[0] if sp.ndim == 2 else 1
        E = np.empty(count, dtype=np.float64)
        Q = np.empty(count, dtype=np.int64) if exact_parts else None
        H = np.empty(count, dtype=np.int64) if exact_parts else None
    ctx.check(ctx.lib.ising_energy(ctx.handle, byref(s), _ptr(sp), count, _ptr(E), _ptr(Q),
                                   _ptr(H), L.MEM_DEVICE if dev else L.MEM_HOST))
    return (E, Q, H) if exact_parts else E


class Server:
    """ising_server_*: continuous batching of independent solves (see the
    header). Requests are copied at submit; results hold the best spins, their
    energy on the full instance and submit / admit / done times (ms)."""

    def __init__(self, ctx: Context, budget_bytes: int, max_active: int = 8,
                 chunk_steps: int = 250, pack: bool = True, helper_threads: int = 0):
        self.ctx = ctx
        cfg = L.ServerCfg()
        cfg.budget_bytes = int(budget_bytes)
        cfg.max_active = int(max_active)
        cfg.chunk_steps = int(chunk_steps)
        cfg.flags = L.SERVER_PACK if pack else 0
        cfg.helper_threads = int(helper_threads)
        self.handle = c_void_p()
        ctx._children.add(self)
        ctx.check(ctx.lib.ising_server_create(ctx.handle, byref(cfg), byref(self.handle)))
        self._n = {}

    def submit(self, inst, restarts, steps, zero_rule=True, target=None, **kw) -> int:
        """Queues a request; with `target` (an energy) it is a time-to-target
        query that finishes once its best energy on the full instance is <=
        target (see ising_server_submit_target)."""
        s, keep = make_instance(inst)
        p = params(restarts, steps, **kw)
        rid = ctypes.c_uint64()
        flags = L.PRUNE_ZERO_RULE if zero_rule else 0
        if target is None:
            self.ctx.check(self.ctx.lib.ising_server_submit(self.handle, byref(s), byref(p), flags,
                                                            byref(rid)))
        else:
            self.ctx.check(self.ctx.lib.ising_server_submit_target(
                self.handle, byref(s), byref(p), flags, float(target), byref(rid)))
        self._n[rid.value] = int(inst.n)
        return rid.value

    def stats(self) -> dict:
        """Where the worker thread's host time went (ising_server_stats_get)."""
        st = L.ServerStats()
        self.ctx.check(self.ctx.lib.ising_server_stats_get(self.handle, byref(st)))
        return {f: getattr(st, f) for f, _ in L.ServerStats._fields_}

    def _result(self, res, rid, spins):
        d = {f: getattr(res, f) for f, _ in L.Result._fields_}
        # (a request cancelled before admission has no spins)
        d["best_spins"] = spins if res.done and res.best_energy == res.best_energy else None
        d["error"] = ""
        if res.done and res.status != 0:
            buf = ctypes.create_string_buffer(512)
            self.ctx.check(self.ctx.lib.ising_server_error(self.handle, rid, buf, 512))
            d["error"] = buf.value.decode(errors="replace")
        return d

    def poll(self, rid: int):
        res = L.Result()
        spins = np.empty(self._n.get(rid, 1), np.int8)
        self.ctx.check(self.ctx.lib.ising_server_poll(self.handle, rid, byref(res), _ptr(spins)))
        return self._result(res, rid, spins)

    def wait(self, rid: int, timeout: float = 600.0):
        res = L.Result()
        spins = np.empty(self._n[rid], np.int8)
        self.ctx.check(self.ctx.lib.ising_server_wait(self.handle, rid, float(timeout), byref(res),
                                                      _ptr(spins)))
        return self._result(res, rid, spins)

    def cancel(self, rid: int):
        """Ends a request early (ising_server_cancel)."""
        self.ctx.check(self.ctx.lib.ising_server_cancel(self.handle, rid))

    def release(self, rid: int):
        self.ctx.check(self.ctx.lib.ising_server_release(self.handle, rid))
        self._n.pop(rid, None)

    def close(self):
        if self.handle:
            self.ctx.lib.ising_server_destroy(self.handle)
            self.handle = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pack:
    """ising_pack_*: sessions of different sizes advanced together, one
    packed step launch and one packed tracking launch per step for all of
    them. The sessions must be tensor-core sessions in the streaming form
    (streaming=True) of one operand type and tile width; each computes what
    it would alone. Close the pack before its sessions."""

    def __init__(self, ctx: Context, sessions):
        self.ctx = ctx
        self.sessions = list(sessions)
        arr = (c_void_p * len(self.sessions))(*[s.handle.value for s in self.sessions])
        self.handle = c_void_p()
        ctx._children.add(self)
        ctx.check(ctx.lib.ising_pack_create(ctx.handle, arr, len(self.sessions), byref(self.handle)))

    def run(self, steps: int):
        self.ctx.check(self.ctx.lib.ising_pack_run(self.handle, int(steps)))

    def close(self):
        if self.handle:
            self.ctx.lib.ising_pack_destroy(self.handle)
            self.handle = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def selftest_waits(ctx: Context, limit_cycles: int):
    """Runs the bounded-wait diagnostic (ising_selftest_waits); returns the
    status code and the mask of waits that gave up, without raising."""
    mask = ctypes.c_int32(-1)
    rc = ctx.lib.ising_selftest_waits(ctx.handle, int(limit_cycles), byref(mask))
    return rc, mask.value


def energy_noalloc(inst, spins, E_out, stream=None):
    """ising_energy_noalloc: energies of spins[count][n] into the caller's
    E_out[count] (all torch CUDA tensors); queues the work on `stream`
    (default: torch's current stream) without allocating anything."""
    torch = _torch()
    lib = L.load()
    s, keep = make_instance(inst)
    if s.mem != L.MEM_DEVICE:
        raise ValueError("energy_noalloc takes a device-memory instance")
    # the C entry point trusts its pointers: check shapes, types and devices
    # here, so that a wrong buffer is an exception and not an out-of-bounds access
    n = int(inst.n)
    if not (isinstance(spins, torch.Tensor) and spins.is_cuda and spins.dtype == torch.int8):
        raise ValueError("spins must be a CUDA int8 tensor")
    if spins.dim() not in (1, 2) or spins.shape[-1] != n or not spins.is_contiguous():
        raise ValueError(f"spins must be contiguous with shape (count, {n}) or ({n},)")
    count = spins.shape[0] if spins.dim() == 2 else 1
    if not (isinstance(E_out, torch.Tensor) and E_out.is_cuda and E_out.dtype == torch.float64
            and E_out.is_contiguous() and E_out.numel() >= count):
        raise ValueError(f"E_out must be a contiguous CUDA float64 tensor of at least {count} elements")
    devs = {spins.device, E_out.device}
    devs |= {a.device for a in keep if isinstance(a, torch.Tensor)}
    if len(devs) != 1:
        raise ValueError("the instance, spins and E_out must be on one device")
    if stream is None:
        stream = torch.cuda.current_stream(spins.device).cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    with torch.cuda.device(spins.device):  # the entry point works on the current device
        rc = lib.ising_energy_noalloc(byref(s), _ptr(spins), count, _ptr(E_out), c_void_p(stream))
    if rc != L.OK:
        msg = lib.ising_energy_noalloc_error()
        raise IsingError(rc, msg.decode() if msg else "")
    return E_out


def _outputs(n, dev):
    """Result buffers on the instance's side: (spins, energy, mem)."""
    if dev:
        torch = _torch()
        return (torch.empty(n, dtype=torch.int8, device="cuda"),
                torch.empty(1, dtype=torch.float64, device="cuda"), L.MEM_DEVICE)
    return np.empty(n, dtype=np.int8), np.empty(1, dtype=np.float64), L.MEM_HOST


def select_domain(ctx: Context, inst, restarts, steps, **kw):
    """One-shot domain selection; returns best spins, energy and stats (on
    the device when the instance is)."""
    s, keep = make_instance(inst)
    p = params(restarts, steps, **kw)
    out, e, mem = _outputs(int(inst.n), s.mem == L.MEM_DEVICE)
    st = L.DSStats()
    ctx.check(ctx.lib.ising_select_domain(ctx.handle, byref(s), byref(p), _ptr(out),
                                          ctypes.cast(_ptr(e), ctypes.POINTER(c_double)),
                                          byref(st), mem))
    return {"best_spins": out, "best_energy": e if mem == L.MEM_DEVICE else float(e[0]),
            **_stats_dict(st)}


def solve(ctx: Context, inst, restarts, steps, zero_rule=True, **kw):
    """Pruning + domain selection + reconstruction + full-instance energy
    (outputs on the device when the instance is)."""
    s, keep = make_instance(inst)
    p = params(restarts, steps, **kw)
    out, e, mem = _outputs(int(inst.n), s.mem == L.MEM_DEVICE)
    st = L.DSStats()
    ctx.check(ctx.lib.ising_solve(ctx.handle, byref(s), byref(p),
                                  L.PRUNE_ZERO_RULE if zero_rule else 0, _ptr(out),
                                  ctypes.cast(_ptr(e), ctypes.POINTER(c_double)), byref(st), mem))
    return {"best_spins": out, "best_energy": e if mem == L.MEM_DEVICE else float(e[0]),
            **_stats_dict(st)}


class Pruned:
    """Result of ising_prune (owned by the library until close())."""

    def __init__(self, ctx: Context, handle: c_void_p, src):
        self.ctx = ctx
        self.handle = handle
        ctx._children.add(self)
        n_red, nnz_red, C, eta, rounds = c_int64(), c_int64(), c_double(), c_double(), c_int32()
        ctx.check(ctx.lib.ising_prune_info(handle, byref(n_red), byref(nnz_red), byref(C),
                                           byref(eta), byref(rounds)))
        self.n = int(src.n)
        self.n_reduced = n_red.value
        self.nnz_reduced = nnz_red.value
        self.constant = C.value
        self.eta = eta.value
        self.rounds = rounds.value
        self._src = src

    def record(self) -> dict:
        n = self.n
        kind = np.empty(n, np.int8)
        rnd = np.empty(n, np.int32)
        value = np.empty(n, np.int8)
        parent = np.empty(n, np.int32)
        sign = np.empty(n, np.int8)
        gidx = np.empty(n, np.int64)
        self.ctx.check(self.ctx.lib.ising_prune_record(self.handle, _ptr(kind), _ptr(rnd),
                                                       _ptr(value), _ptr(parent), _ptr(sign),
                                                       _ptr(gidx), L.MEM_HOST))
        return dict(kind=kind, round=rnd, value=value, parent=parent, sign=sign, g_index=gidx)

    def reduced(self):
        """Reduced instance copied to host numpy arrays (same attributes as the input)."""
        from types import SimpleNamespace
        src = self._src
        dense = src.layout == "dense"
        jd = np.asarray(src.J if dense else src.data)
        if _is_torch(jd):
            jd = jd.cpu().numpy()
        nr, nz = self.n_reduced, self.nnz_reduced
        J = np.empty(nr * nr if dense else nz, dtype=jd.dtype)
        ip = None if dense else np.empty(nr + 1, np.int64)
        ix = None if dense else np.empty(nz, np.int32)
        h = np.empty(nr, np.float64)
        self.ctx.check(self.ctx.lib.ising_prune_reduced_copy(self.handle, _ptr(J), _ptr(ip),
                                                             _ptr(ix), _ptr(h), L.MEM_HOST))
        return SimpleNamespace(n=nr, layout=src.layout, J=J.reshape(nr, nr) if dense else None,
                               indptr=ip, indices=ix, data=None if dense else J, h=h,
                               j_scale=src.j_scale, convention=src.convention)

    def reconstruct(self, reduced_spins) -> np.ndarray:
        sg = _host(reduced_spins, np.int8)
        out = np.empty(self.n, np.int8)
        self.ctx.check(self.ctx.lib.ising_reconstruct(self.ctx.handle, self.handle, _ptr(sg),
                                                      _ptr(out), L.MEM_HOST))
        return out

    def close(self):
        if self.handle:
            self.ctx.lib.ising_prune_free(self.handle)
            self.handle = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def prune(ctx: Context, inst, zero_rule: bool = True) -> Pruned:
    s, keep = make_instance(inst)
    h = c_void_p()
    ctx.check(ctx.lib.ising_prune(ctx.handle, byref(s), L.PRUNE_ZERO_RULE if zero_rule else 0,
                                  byref(h)))
    return Pruned(ctx, h, inst)


class Session:
    """ising_ds_* session: create, run, inspect, finish."""

    def __init__(self, ctx: Context, inst, restarts, steps, **kw):
        self.ctx = ctx
        s, keep = make_instance(inst)
        self.p = params(restarts, steps, **kw)
        self.n = int(inst.n)
        self.B = int(restarts)
        self.handle = c_void_p()
        ctx._children.add(self)
        ctx.check(ctx.lib.ising_ds_create(ctx.handle, byref(s), byref(self.p), byref(self.handle)))

    def run(self, steps: int):
        self.ctx.check(self.ctx.lib.ising_ds_run(self.handle, int(steps)))

    def finish(self):
        self.ctx.check(self.ctx.lib.ising_ds_finish(self.handle))

    def export_state(self):
        B, n = self.B, self.n
        th = np.empty((B, n), np.float32)
        m = np.empty((B, n), np.float32)
        v = np.empty((B, n), np.float32)
        sp = np.empty((B, n), np.int8)
        t = c_int64()
        self.ctx.check(self.ctx.lib.ising_ds_export_state(self.handle, _ptr(th), _ptr(m), _ptr(v),
                                                          _ptr(sp), byref(t), L.MEM_HOST))
        return dict(theta=th, m=m, v=v, spins=sp, t=t.value)

    def import_state(self, theta, m, v, t: int):
        th = _host(theta, np.float32)
        mm = _host(m, np.float32)
        vv = _host(v, np.float32)
        self.ctx.check(self.ctx.lib.ising_ds_import_state(self.handle, _ptr(th), _ptr(mm),
                                                          _ptr(vv), int(t), L.MEM_HOST))

    def coupling(self) -> np.ndarray:
        """G = J s of the next step's spins, [B][n] float32."""
        G = np.empty((self.B, self.n), np.float32)
        self.ctx.check(self.ctx.lib.ising_ds_coupling(self.handle, _ptr(G), L.MEM_HOST))
        return G

    def trace(self) -> np.ndarray:
        """Per-CTA role timeline of the last profiled step launch, (CTAs, 8) ns."""
        cnt = c_int64()
        self.ctx.check(self.ctx.lib.ising_ds_trace(self.handle, None, 0, byref(cnt)))
        out = np.zeros(max(cnt.value, 0), np.uint64)
        if cnt.value:
            self.ctx.check(self.ctx.lib.ising_ds_trace(self.handle, _ptr(out), cnt.value,
                                                       byref(cnt)))
        return out.reshape(-1, 8)

    def last_energies(self) -> np.ndarray:
        E = np.empty(self.B, np.float64)
        self.ctx.check(self.ctx.lib.ising_ds_last_energies(self.handle, _ptr(E), L.MEM_HOST))
        return E

    def set_tiles(self, restarts_per_tile: int, pair: int = 0):
        """Tensor-core streaming form: tile width and CTA pairs (0 none, 1
        sharing spin tiles by multicast, 2 one MMA per pair; see
        ising_ds_set_tiles)."""
        self.ctx.check(self.ctx.lib.ising_ds_set_tiles(self.handle, int(restarts_per_tile),
                                                       int(pair)))

    def work(self) -> int:
        """Restart-steps the update launches computed (below B x steps when
        the convergence rule retires restarts)."""
        w = c_int64()
        self.ctx.check(self.ctx.lib.ising_ds_work(self.handle, byref(w)))
        return w.value

    def convergence(self) -> np.ndarray:
        """Step at which each restart stopped under the convergence rule (0
        while it runs)."""
        out = np.empty(self.B, np.int64)
        self.ctx.check(self.ctx.lib.ising_ds_convergence(self.handle, _ptr(out), L.MEM_HOST))
        return out

    def restart_best(self, device: bool = False):
        """Per-restart best energy, step and spins [B][n]; torch tensors on
        the session's device when `device`, else numpy arrays."""
        if device:
            torch = _torch()
            dev = torch.device("cuda", self.ctx.device)
            E = torch.empty(self.B, dtype=torch.float64, device=dev)
            st = torch.empty(self.B, dtype=torch.int64, device=dev)
            sp = torch.empty((self.B, self.n), dtype=torch.int8, device=dev)
            mem = L.MEM_DEVICE
        else:
            E = np.empty(self.B, np.float64)
            st = np.empty(self.B, np.int64)
            sp = np.empty((self.B, self.n), np.int8)
            mem = L.MEM_HOST
        self.ctx.check(self.ctx.lib.ising_ds_restart_best(self.handle, _ptr(E), _ptr(st),
                                                          _ptr(sp), mem))
        return E, st, sp

    def result(self):
        out = np.empty(self.n, np.int8)
        e = c_double()
        st = L.DSStats()
        self.ctx.check(self.ctx.lib.ising_ds_result(self.handle, _ptr(out), byref(e), byref(st),
                                                    L.MEM_HOST))
        return {"best_spins": out, "best_energy": e.value, **_stats_dict(st)}

    def close(self):
        if self.handle:
            self.ctx.lib.ising_ds_destroy(self.handle)
            self.handle = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
