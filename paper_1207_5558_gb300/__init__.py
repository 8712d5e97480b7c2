"""GB300-native directional SLSHT (Khalid et al., arXiv:1207.5558).

A thin Python layer over libslsht (include/slsht.h).  The functions keep the
C names; ``Context`` bundles a context handle with convenience marshalling of
torch tensors / numpy arrays.  PyTorch is used only for device memory and
streams.  The CUDA library must be built (``__graft_entry__.build()``): there
is no CPU fallback, and every call raises if the library is missing.
"""
import ctypes

from . import _abi
from ._abi import (SLSHT_FP32_BULK, SLSHT_FP64, SLSHT_OPT_ALPHA_ENGINE,  # noqa: F401
                   SLSHT_OPT_BETA_ROUTE, SLSHT_OPT_CHUNK_PAIRS, SLSHT_OPT_GAUNT_TABLE, SLSHT_OPT_WAIT_TEST, SLSHT_OPT_REAL_FIELDS,
                   SLSHT_OPT_COUPLING, SLSHT_OPT_FP64_ARITH, SLSHT_OPT_WINDOW_ORDERS, SLSHT_OPT_ROTWIN_ENGINE,
                   SLSHT_BATCH_NO_GRAPH, SLSHT_BATCH_NO_TUNE, SLSHT_BATCH_NO_TC, SLSHT_BATCH_NO_DD,
                   SLSHT_BATCH_FP64_DD,
                   SLSHT_BQ_TILE_COLS, SLSHT_BQ_ALPHA_FORM, SLSHT_BQ_TUNED, SLSHT_BQ_TILES, SLSHT_BQ_KERNELS,
                   SLSHT_BQ_GRAPH, SLSHT_BQ_BYTES, SLSHT_BQ_SAMPLES, SLSHT_BQ_ENGINE,
                   SlshtError, STAGE_NAMES,
                   slsht_batch_item, slsht_desc, slsht_stats)

__all__ = ["Context", "make_desc", "SLSHT_FP64", "SLSHT_FP32_BULK", "SlshtError",
           "slsht_create", "slsht_destroy", "slsht_forward", "slsht_forward_noalloc", "slsht_forward_windows",
           "slsht_window_ellipse", "slsht_batch_create", "slsht_batch_launch", "slsht_batch_query",
           "slsht_batch_destroy", "slsht_tune", "Batch",
           "slsht_inverse", "slsht_inverse_alt", "slsht_steer_gamma", "slsht_submit",
           "slsht_poll", "slsht_poll_times", "slsht_drain", "slsht_strerror", "slsht_check_args", "slsht_profile",
           "slsht_get_stats", "slsht_set_option", "slsht_mem_used", "slsht_version"]


def make_desc(L_f, L_h, grid, prec=SLSHT_FP64):
    na, nb, ng = grid
    return slsht_desc(int(L_f), int(L_h), int(na), int(nb), int(ng), int(prec))


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# ------------------------------------------------------------ C-named calls
def slsht_create(device=0, mem_budget_bytes=0):
    lib = _abi.load()
    h = ctypes.c_void_p()
    _abi.check(lib.slsht_create(ctypes.byref(h), int(device), int(mem_budget_bytes)), "slsht_create")
    return h


def slsht_destroy(ctx):
    _abi.load().slsht_destroy(ctx)


def slsht_forward(ctx, desc, f_lm, h_lm, lm, n_pairs, g_out, stream=None):
    return _abi.check(_abi.load().slsht_forward(ctx, ctypes.byref(desc), _abi.ptr(f_lm), _abi.ptr(h_lm),
                                                _abi.ptr(lm), int(n_pairs), _abi.ptr(g_out),
                                                _stream(stream)), "slsht_forward")


def slsht_forward_windows(ctx, desc, f_lm, n_windows, h_lms, lm, n_pairs, g_out, stream=None):
    return _abi.check(_abi.load().slsht_forward_windows(ctx, ctypes.byref(desc), _abi.ptr(f_lm), int(n_windows),
                                                        _abi.ptr(h_lms), _abi.ptr(lm), int(n_pairs),
                                                        _abi.ptr(g_out), _stream(stream)),
                      "slsht_forward_windows")


def slsht_window_ellipse(ctx, L, theta_c, a, h_out, n_phi=0, n_theta=0, stream=None):
    """Concentrated window of R(theta_c, a) into h_out (complex128 [L*L]);
    returns the concentration."""
    lam = ctypes.c_double()
    _abi.check(_abi.load().slsht_window_ellipse(ctx, int(L), float(theta_c), float(a), int(n_phi), int(n_theta),
                                                _abi.ptr(h_out), ctypes.byref(lam), _stream(stream)),
               "slsht_window_ellipse")
    return lam.value


def slsht_inverse(ctx, desc, g_in, h00, lm, n_pairs, f_out, stream=None):
    hv = (ctypes.c_double * 2)(float(complex(h00).real), float(complex(h00).imag))
    return _abi.check(_abi.load().slsht_inverse(ctx, ctypes.byref(desc), _abi.ptr(g_in), hv, _abi.ptr(lm),
                                                int(n_pairs), _abi.ptr(f_out), _stream(stream)),
                      "slsht_inverse")


def slsht_inverse_alt(ctx, desc, g_in, h_lm, lm_in, n_in, p, lm_out, n_out, f_out, stream=None):
    return _abi.check(_abi.load().slsht_inverse_alt(ctx, ctypes.byref(desc), _abi.ptr(g_in), _abi.ptr(h_lm),
                                                    _abi.ptr(lm_in), int(n_in), int(p), _abi.ptr(lm_out),
                                                    int(n_out), _abi.ptr(f_out), _stream(stream)),
                      "slsht_inverse_alt")


def slsht_steer_gamma(ctx, desc, g_in, n_pairs, gammas, n_g, Q, g_out, stream=None):
    return _abi.check(_abi.load().slsht_steer_gamma(ctx, ctypes.byref(desc), _abi.ptr(g_in), int(n_pairs),
                                                    _abi.ptr(gammas), int(n_g), int(Q), _abi.ptr(g_out),
                                                    _stream(stream)), "slsht_steer_gamma")


def slsht_forward_noalloc(desc, f_lm, h_lm, lm, n_pairs, g_out, stream=None):
    """slsht_forward without a context and without device allocation (static
    scratch of SLSHT_NOALLOC_SCRATCH_BYTES); g_out must be device memory."""
    return _abi.check(_abi.load().slsht_forward_noalloc(ctypes.byref(desc), _abi.ptr(f_lm), _abi.ptr(h_lm),
                                                        _abi.ptr(lm), int(n_pairs), _abi.ptr(g_out),
                                                        _stream(stream)), "slsht_forward_noalloc")


def slsht_batch_create(ctx, items, flags=0, stream=None):
    """items: a ctypes array of slsht_batch_item.  Returns the plan handle."""
    h = ctypes.c_void_p()
    _abi.check(_abi.load().slsht_batch_create(ctx, len(items), items, int(flags), _stream(stream), ctypes.byref(h)),
               "slsht_batch_create")
    return h


def slsht_batch_launch(batch, stream=None):
    return _abi.check(_abi.load().slsht_batch_launch(batch, _stream(stream)), "slsht_batch_launch")


def slsht_batch_query(batch, item, what):
    v = ctypes.c_int64()
    _abi.check(_abi.load().slsht_batch_query(batch, int(item), int(what), ctypes.byref(v)), "slsht_batch_query")
    return v.value


def slsht_batch_destroy(batch):
    _abi.load().slsht_batch_destroy(batch)


def slsht_tune(ctx, desc):
    return _abi.check(_abi.load().slsht_tune(ctx, ctypes.byref(desc)), "slsht_tune")


def slsht_submit(ctx, desc, f_lm, h_lm, lm, n_pairs, g_out):
    t = ctypes.c_uint64()
    _abi.check(_abi.load().slsht_submit(ctx, ctypes.byref(desc), _abi.ptr(f_lm), _abi.ptr(h_lm),
                                        _abi.ptr(lm), int(n_pairs), _abi.ptr(g_out), ctypes.byref(t)),
               "slsht_submit")
    return t.value


def slsht_poll(ctx, ticket):
    return _abi.load().slsht_poll(ctx, ctypes.c_uint64(ticket))


def slsht_poll_times(ctx, ticket):
    """(status, times): times = [queue, host issue, device, total] in ms once
    the request has finished, else None."""
    t = (ctypes.c_double * 4)()
    s = _abi.load().slsht_poll_times(ctx, ctypes.c_uint64(ticket), ctypes.cast(t, ctypes.c_void_p))
    return s, (list(t) if s != 1 else None)


def slsht_drain(ctx, timeout_ms=60000):
    return _abi.check(_abi.load().slsht_drain(ctx, int(timeout_ms)), "slsht_drain")


def slsht_strerror(code):
    return _abi.load().slsht_strerror(int(code)).decode()


def slsht_check_args(desc, lm_host, n_pairs):
    return _abi.load().slsht_check_args(ctypes.byref(desc), _abi.ptr(lm_host), int(n_pairs))


def slsht_profile(ctx, enable):
    return _abi.check(_abi.load().slsht_profile(ctx, int(bool(enable))), "slsht_profile")


def slsht_get_stats(ctx, reset=False):
    s = slsht_stats()
    _abi.check(_abi.load().slsht_get_stats(ctx, ctypes.byref(s), int(bool(reset))), "slsht_get_stats")
    return {"launches": {n: int(s.launches[i]) for i, n in enumerate(STAGE_NAMES)},
            "ms": {n: float(s.ms[i]) for i, n in enumerate(STAGE_NAMES)},
            "samples_written": int(s.samples_written)}


def slsht_set_option(ctx, option, value):
    return _abi.check(_abi.load().slsht_set_option(ctx, int(option), int(value)), "slsht_set_option")


def slsht_mem_used(ctx):
    return int(_abi.load().slsht_mem_used(ctx))


def slsht_version():
    return _abi.load().slsht_version().decode()


# ------------------------------------------------------------ convenience
class Context:
    """One libslsht context on one CUDA device."""

    def __init__(self, device=0, mem_budget_bytes=0):
        self.device = device
        self.h = slsht_create(device, mem_budget_bytes)

    def close(self):
        if self.h is not None:
            slsht_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, option, value):
        slsht_set_option(self.h, option, value)

    def forward(self, L_f, L_h, grid, f, h, lm, prec=SLSHT_FP64, g_out=None, stream=None):
        """g(rho; l, m) for the pairs in lm ([n, 2] int32).  f, h: complex128
        (numpy on the host or torch on the device).  Returns g_out (a new
        torch tensor [n, Na, Nb, Ng] on the device when not given)."""
        import numpy as np
        import torch
        lm = _as_pairs(lm)
        n = int(lm.shape[0])
        if g_out is None:
            dt = torch.complex128 if prec == SLSHT_FP64 else torch.complex64
            g_out = torch.empty((n,) + tuple(grid), dtype=dt, device="cuda:%d" % self.device)
        f = _as_c128(f)
        h = _as_c128(h)
        slsht_forward(self.h, make_desc(L_f, L_h, grid, prec), f, h, lm, n, g_out, stream)
        _ = np
        return g_out

    def forward_windows(self, L_f, L_h, grid, f, hs, lm, prec=SLSHT_FP64, g_out=None, stream=None):
        """g for several windows hs ([n_windows, L_h^2] complex128) over one
        signal: the coupling is formed once.  Returns g_out
        [n_windows, n, Na, Nb, Ng] (a new device tensor when not given)."""
        import torch
        lm = _as_pairs(lm)
        n = int(lm.shape[0])
        hs = _as_c128(hs)
        nw = int(hs.shape[0])
        if g_out is None:
            dt = torch.complex128 if prec == SLSHT_FP64 else torch.complex64
            g_out = torch.empty((nw, n) + tuple(grid), dtype=dt, device="cuda:%d" % self.device)
        slsht_forward_windows(self.h, make_desc(L_f, L_h, grid, prec), _as_c128(f), nw, hs, lm, n, g_out, stream)
        return g_out

    def window_ellipse(self, L, theta_c, a, n_phi=0, n_theta=0):
        """(h, concentration): the most concentrated window of R(theta_c, a)
        at band limit L, computed on the device (h: host complex128 [L*L])."""
        import numpy as np
        h = np.zeros(L * L, dtype=np.complex128)
        lam = slsht_window_ellipse(self.h, L, theta_c, a, h, n_phi, n_theta)
        return h, lam

    def inverse(self, L_f, L_h, grid, g, h00, lm, prec=SLSHT_FP64, f_out=None, stream=None):
        """f_lm for each pair from g (device tensor).  Returns a host numpy
        complex128 array unless f_out is given."""
        import numpy as np
        lm = _as_pairs(lm)
        n = int(lm.shape[0])
        host = f_out is None
        if host:
            f_out = np.zeros(n, dtype=np.complex128)
        slsht_inverse(self.h, make_desc(L_f, L_h, grid, prec), g, h00, lm, n, f_out, stream)
        if host:
            import torch
            torch.cuda.synchronize(self.device)
        return f_out

    def inverse_alt(self, L_f, L_h, grid, g, h, lm_in, p, lm_out, prec=SLSHT_FP64, stream=None):
        """f_lm for the pairs lm_out from g (device tensor, rows lm_in) without
        h_0^0 (slsht_inverse_alt, window degree p).  Returns host complex128."""
        import numpy as np
        lm_in = _as_pairs(lm_in)
        lm_out = _as_pairs(lm_out)
        f_out = np.zeros(int(lm_out.shape[0]), dtype=np.complex128)
        slsht_inverse_alt(self.h, make_desc(L_f, L_h, grid, prec), g, _as_c128(h), lm_in, int(lm_in.shape[0]), p,
                          lm_out, int(lm_out.shape[0]), f_out, stream)
        return f_out

    def submit(self, L_f, L_h, grid, f, h, lm, g_out, prec=SLSHT_FP64):
        lm = _as_pairs(lm)
        return slsht_submit(self.h, make_desc(L_f, L_h, grid, prec), _as_c128(f), _as_c128(h), lm,
                            int(lm.shape[0]), g_out)

    def poll(self, ticket):
        return slsht_poll(self.h, ticket)

    def poll_times(self, ticket):
        """(status, [queue, host issue, device, total] ms or None)."""
        return slsht_poll_times(self.h, ticket)

    def drain(self, timeout_ms=60000):
        return slsht_drain(self.h, timeout_ms)

    def profile(self, enable=True):
        slsht_profile(self.h, enable)

    def stats(self, reset=False):
        return slsht_get_stats(self.h, reset)

    def mem_used(self):
        return slsht_mem_used(self.h)

    def tune(self, L_f, L_h, grid, prec=SLSHT_FP64):
        """Measure and cache the tile shapes of one grid shape (slsht_tune)."""
        slsht_tune(self.h, make_desc(L_f, L_h, grid, prec))

    def batch(self, items, flags=0, stream=None):
        """A Batch plan over `items` (see Batch)."""
        return Batch(self, items, flags, stream)


class Batch:
    """A batch plan over several analyses of one context.

    items: a list of dicts with keys L_f, L_h, grid (N_alpha, N_beta, N_gamma),
    f and h (complex128 DEVICE tensors), lm ([n, 2] pairs) and optional prec
    and g_out (a device tensor; allocated when absent).  The plan keeps
    references to f, h and g_out: every launch() reads what f and h hold then
    and writes g_out (see slsht_batch_create).  outputs: the g_out tensors."""

    def __init__(self, ctx, items, flags=0, stream=None):
        import torch
        self.ctx = ctx
        self.h = None
        self.keep = []
        self.outputs = []
        arr = (slsht_batch_item * len(items))()
        for i, it in enumerate(items):
            prec = it.get("prec", SLSHT_FP64)
            lm = _as_pairs(it["lm"])
            n = int(lm.shape[0])
            g = it.get("g_out")
            if g is None:
                dt = torch.complex128 if prec == SLSHT_FP64 else torch.complex64
                g = torch.empty((n,) + tuple(it["grid"]), dtype=dt, device="cuda:%d" % ctx.device)
            f, h = it["f"], it["h"]
            self.keep += [f, h, lm, g]
            self.outputs.append(g)
            arr[i].desc = make_desc(it["L_f"], it["L_h"], it["grid"], prec)
            arr[i].f_lm = f.data_ptr()
            arr[i].h_lm = h.data_ptr()
            arr[i].lm = _abi.ptr(lm).value
            arr[i].n_pairs = n
            arr[i].g_out = g.data_ptr()
        self.h = slsht_batch_create(ctx.h, arr, flags, stream)

    def launch(self, stream=None):
        slsht_batch_launch(self.h, stream)

    def query(self, what, item=0):
        return slsht_batch_query(self.h, item, what)

    def close(self):
        # a plan dies with its context: after Context.close() only drop the handle
        if self.h is not None and self.ctx.h is not None:
            slsht_batch_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _as_pairs(lm):
    import numpy as np
    if hasattr(lm, "data_ptr") and getattr(lm, "is_cuda", False):
        return lm
    return np.ascontiguousarray(np.asarray(lm, dtype=np.int32).reshape(-1, 2))


def _as_c128(x):
    import numpy as np
    if hasattr(x, "data_ptr"):
        return x.contiguous()
    return np.ascontiguousarray(np.asarray(x, dtype=np.complex128))
