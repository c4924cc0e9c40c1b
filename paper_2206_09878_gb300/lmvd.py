"""Thin Python binding of liblmvd (include/lmvd.h): argument marshalling only.

Every function has the name of the C entry point it calls. Array arguments are torch tensors
(CUDA device memory, or host memory -- pinned for asynchronous copies) with the layouts of
lmvd.h: complex128 [y][kz][kx] spectral arrays, float64 plane means. No computation happens
here; if the compiled library is missing this module raises ImportError instead of falling back.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# LMVD_LIBRARY selects another build of the same library, e.g. the index-checked liblmvd_check.so
LIB_PATH = os.environ.get("LMVD_LIBRARY") or os.path.join(_HERE, "liblmvd.so")

LMVD_FIELD_RZ = 0
LMVD_FIELD_ZDOT = 1
LMVD_FIELD_RHO_T = 2
LMVD_FIELD_MC1 = 3
LMVD_FIELD_MC2 = 4
LMVD_FIELD_MC3 = 5
LMVD_FIELD_R_OMEGA2 = 6
LMVD_FIELD_R_PHI2 = 7
LMVD_FIELD_R_MEANS = 8


class lmvd_config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("spline_order", ctypes.c_int),
                ("lx", ctypes.c_double), ("lz", ctypes.c_double), ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("re", ctypes.c_double), ("sc", ctypes.c_double), ("fr", ctypes.c_double),
                ("rho_heavy", ctypes.c_double), ("rho_light", ctypes.c_double),
                ("dt", ctypes.c_double), ("kf", ctypes.c_int), ("beta_n", ctypes.c_double),
                ("beta_p", ctypes.c_double), ("n_startup", ctypes.c_int), ("precision", ctypes.c_int),
                ("bc_mode", ctypes.c_int), ("memory_layout", ctypes.c_int)]


class LmvdError(RuntimeError):
    def __init__(self, code, where):
        super().__init__("%s failed: %s (%d)" % (where, lmvd_strerror(code), code))
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("liblmvd.so is not built (%s); run paper_2206_09878_gb300.build.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    sig = {
        "lmvd_default_config": (I, [ctypes.POINTER(lmvd_config), I, I, I]),
        "lmvd_create": (I, [ctypes.POINTER(lmvd_config), P, ctypes.POINTER(P)]),
        "lmvd_destroy": (None, [P]),
        "lmvd_set_state": (I, [P, P, P, P, P, P, P]),
        "lmvd_get_state": (I, [P, P, P, P, P, P, P]),
        "lmvd_history_bytes": (S, [P]),
        "lmvd_advance_substage": (I, [P]),
        "lmvd_step": (I, [P, I]),
        "lmvd_get_field": (I, [P, I, P]),
        "lmvd_field_bytes": (S, [P, I]),
        "lmvd_substage_index": (I, [P]),
        "lmvd_synchronize": (I, [P]),
        "lmvd_status": (I, [P]),
        "lmvd_strerror": (ctypes.c_char_p, [I]),
        "lmvd_profile_enable": (I, [P, I]),
        "lmvd_profile_read": (I, [P, I, ctypes.POINTER(ctypes.c_double)]),
        "lmvd_kernel_class_name": (ctypes.c_char_p, [I]),
        "lmvd_kernel_launches": (ctypes.c_longlong, [P]),
        "lmvd_inverse_transform": (I, [P, P, P, I]),
        "lmvd_forward_transform": (I, [P, P, P, I]),
        "lmvd_inverse_transform_noalloc": (I, [I, I, I, P, P, I, P]),
        "lmvd_state_bytes": (S, [P]),
        "lmvd_adjoint_substage": (I, [P, P, P, P, P]),
        "lmvd_adjoint_startup": (I, [P, P, P, P]),
        "lmvd_device_bytes": (S, [P]),
        "lmvd_diagnostics_enable": (I, [P, I]),
        "lmvd_diagnostics": (I, [P, ctypes.POINTER(ctypes.c_double), I]),
        "lmvd_graphs_enable": (I, [P, I]),
        "lmvd_graph_count": (I, [P]),
        "lmvd_df64_convert": (I, [P, P, P, P, P, P, S, P]),
        "lmvd_checked_build": (I, []),
        "lmvd_rate_probe": (I, [I, I, ctypes.POINTER(ctypes.c_double), P]),
        "lmvd_tile_wait_probe": (I, [P, I, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _ = D
    return lib


_lib = _load()

EXPORTED = ("lmvd_default_config", "lmvd_create", "lmvd_destroy", "lmvd_set_state", "lmvd_get_state",
            "lmvd_history_bytes", "lmvd_advance_substage", "lmvd_step", "lmvd_get_field", "lmvd_field_bytes",
            "lmvd_substage_index", "lmvd_synchronize", "lmvd_status", "lmvd_strerror", "lmvd_profile_enable",
            "lmvd_profile_read", "lmvd_kernel_class_name", "lmvd_kernel_launches", "lmvd_inverse_transform",
            "lmvd_forward_transform", "lmvd_inverse_transform_noalloc", "lmvd_state_bytes",
            "lmvd_adjoint_substage", "lmvd_adjoint_startup", "lmvd_device_bytes", "lmvd_diagnostics_enable",
            "lmvd_diagnostics", "lmvd_graphs_enable", "lmvd_graph_count", "lmvd_df64_convert",
            "lmvd_checked_build", "lmvd_rate_probe", "lmvd_tile_wait_probe")
LMVD_KERNEL_CLASSES = 13


def _ptr(t):
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("arrays passed to liblmvd must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _check(code, where):
    if code != 0:
        raise LmvdError(code, where)
    return code


def lmvd_strerror(code):
    return _lib.lmvd_strerror(int(code)).decode()


def lmvd_default_config(nx, ny, nz, **overrides):
    cfg = lmvd_config()
    _check(_lib.lmvd_default_config(ctypes.byref(cfg), nx, ny, nz), "lmvd_default_config")
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise KeyError(k)
        setattr(cfg, k, v)
    return cfg


def lmvd_create(cfg, stream=None):
    """Returns an opaque context handle (ctypes.c_void_p). stream: torch.cuda.Stream or None (current)."""
    if stream is None:
        stream = torch.cuda.current_stream()
    h = ctypes.c_void_p()
    _check(_lib.lmvd_create(ctypes.byref(cfg), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h)), "lmvd_create")
    return h


def lmvd_destroy(h):
    _lib.lmvd_destroy(h)


def lmvd_set_state(h, z, om, m2, mm1, mm3, history=None):
    _check(_lib.lmvd_set_state(h, _ptr(z), _ptr(om), _ptr(m2), _ptr(mm1), _ptr(mm3), _ptr(history)),
           "lmvd_set_state")


def lmvd_get_state(h, z=None, om=None, m2=None, mm1=None, mm3=None, history=None):
    _check(_lib.lmvd_get_state(h, _ptr(z), _ptr(om), _ptr(m2), _ptr(mm1), _ptr(mm3), _ptr(history)),
           "lmvd_get_state")


def lmvd_history_bytes(h):
    return int(_lib.lmvd_history_bytes(h))


def lmvd_advance_substage(h):
    _check(_lib.lmvd_advance_substage(h), "lmvd_advance_substage")


def lmvd_step(h, nsteps):
    _check(_lib.lmvd_step(h, int(nsteps)), "lmvd_step")


def lmvd_field_bytes(h, which):
    return int(_lib.lmvd_field_bytes(h, int(which)))


def lmvd_get_field(h, which, out):
    _check(_lib.lmvd_get_field(h, int(which), _ptr(out)), "lmvd_get_field")


def lmvd_substage_index(h):
    return int(_lib.lmvd_substage_index(h))


def lmvd_synchronize(h):
    _check(_lib.lmvd_synchronize(h), "lmvd_synchronize")


def lmvd_status(h):
    return int(_lib.lmvd_status(h))


def lmvd_profile_enable(h, on=True):
    _check(_lib.lmvd_profile_enable(h, 1 if on else 0), "lmvd_profile_enable")


def lmvd_profile_read(h, cls):
    """(total_ms, launches, algorithmic_flops, algorithmic_bytes) of one kernel class."""
    out = (ctypes.c_double * 4)()
    _check(_lib.lmvd_profile_read(h, int(cls), out), "lmvd_profile_read")
    return tuple(out)


def lmvd_kernel_class_name(cls):
    return _lib.lmvd_kernel_class_name(int(cls)).decode()


def lmvd_kernel_launches(h):
    return int(_lib.lmvd_kernel_launches(h))


def lmvd_inverse_transform(h, spec, phys, nfields):
    _check(_lib.lmvd_inverse_transform(h, _ptr(spec), _ptr(phys), int(nfields)), "lmvd_inverse_transform")


def lmvd_forward_transform(h, phys, spec, nfields):
    _check(_lib.lmvd_forward_transform(h, _ptr(phys), _ptr(spec), int(nfields)), "lmvd_forward_transform")


def lmvd_inverse_transform_noalloc(nx, ny, nz, spec, phys, nfields, stream=None):
    """Context-free synthesis that allocates no device memory (static per-device working array)."""
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(_lib.lmvd_inverse_transform_noalloc(int(nx), int(ny), int(nz), _ptr(spec), _ptr(phys), int(nfields),
                                               ctypes.c_void_p(stream.cuda_stream)),
           "lmvd_inverse_transform_noalloc")


def lmvd_checked_build():
    """1 if the loaded library is the index-checked build (liblmvd_check.so), else 0."""
    return int(_lib.lmvd_checked_build())


def lmvd_rate_probe(op, iters=20000, stream=None):
    """Operations per second of op (0 FP64 FMA, 1 FP64 add, 2 FP64 multiply, 3 FP32 FMA) on the current device."""
    out = ctypes.c_double(0.0)
    st = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    _check(_lib.lmvd_rate_probe(int(op), int(iters), ctypes.byref(out), st), "lmvd_rate_probe")
    return out.value


def lmvd_tile_wait_probe(src, extra_bytes, status, stream=None):
    """The transforms' bounded tile-copy wait on its own: src a CUDA float64 tensor (>= 16 values), status a
    CUDA int32 tensor of one element (bit 2: the wait gave up; bit 3: the copied data differ)."""
    st = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    _check(_lib.lmvd_tile_wait_probe(_ptr(src), int(extra_bytes), _ptr(status), st), "lmvd_tile_wait_probe")


def lmvd_state_bytes(h):
    return int(_lib.lmvd_state_bytes(h))


def lmvd_adjoint_substage(h, state_bar_out, history_bar_out, state_bar_in, history_bar_in):
    _check(_lib.lmvd_adjoint_substage(h, _ptr(state_bar_out), _ptr(history_bar_out), _ptr(state_bar_in),
                                      _ptr(history_bar_in)), "lmvd_adjoint_substage")


def lmvd_graphs_enable(h, on=True):
    _check(_lib.lmvd_graphs_enable(h, 1 if on else 0), "lmvd_graphs_enable")


def lmvd_df64_convert(x, hi, lo, pair_hi, pair_lo, out_sum, stream=None):
    """Device conversions of the precision path on caller tensors (see lmvd.h)."""
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(_lib.lmvd_df64_convert(_ptr(x), _ptr(hi), _ptr(lo), _ptr(pair_hi), _ptr(pair_lo), _ptr(out_sum),
                                  int(x.numel()), ctypes.c_void_p(stream.cuda_stream)), "lmvd_df64_convert")


def lmvd_graph_count(h):
    return int(_lib.lmvd_graph_count(h))


def lmvd_diagnostics_enable(h, on=True):
    _check(_lib.lmvd_diagnostics_enable(h, 1 if on else 0), "lmvd_diagnostics_enable")


def lmvd_diagnostics(h):
    """dict(substage, mass_residual, fp_changes=[...], kinetic_energy, max_momentum, mean_m2c_y0) of the last
    substage's record."""
    buf = (ctypes.c_double * 24)()
    n = _lib.lmvd_diagnostics(h, buf, 24)
    if n < 0:
        _check(n, "lmvd_diagnostics")
    vals = list(buf)[:min(n, 24)]
    return dict(substage=int(vals[0]), mass_residual=vals[1], fp_changes=vals[2:-3], kinetic_energy=vals[-3],
                max_momentum=vals[-2], mean_m2c_y0=vals[-1])


def lmvd_device_bytes(h):
    return int(_lib.lmvd_device_bytes(h))


def lmvd_adjoint_startup(h, state_bar_out, history_bar_out, state_bar_in):
    _check(_lib.lmvd_adjoint_startup(h, _ptr(state_bar_out), _ptr(history_bar_out), _ptr(state_bar_in)),
           "lmvd_adjoint_startup")


# ---------------------------------------------------------------- convenience (still marshalling only)
class Context:
    """Owns one lmvd context plus torch buffers shaped for its state; frees the context on close()."""

    def __init__(self, cfg, device="cuda", stream=None):
        self.cfg = cfg
        self.device = torch.device(device)
        self.stream = torch.cuda.current_stream() if stream is None else stream
        self.h = lmvd_create(cfg, self.stream)
        nxh = cfg.nx // 2 + 1
        self.shape = (cfg.ny, cfg.nz, nxh)
        self.shape_m2 = (cfg.ny + 1, cfg.nz, nxh)

    def empty_state(self, device=None, pin=False):
        dev = self.device if device is None else torch.device(device)
        kw = dict(device=dev)
        if pin and dev.type == "cpu":
            kw["pin_memory"] = True
        return dict(z=torch.zeros(self.shape, dtype=torch.complex128, **kw),
                    om=torch.zeros(self.shape, dtype=torch.complex128, **kw),
                    m2=torch.zeros(self.shape_m2, dtype=torch.complex128, **kw),
                    mm1=torch.zeros(self.cfg.ny, dtype=torch.float64, **kw),
                    mm3=torch.zeros(self.cfg.ny, dtype=torch.float64, **kw))

    # Stream order between torch and the library: tensors handed to the library were produced on torch's
    # current stream, so the context's stream waits for it first (wait_inputs); tensors the library writes
    # are read on torch's current stream, which waits for the context's stream afterwards (publish).
    def wait_inputs(self):
        cur = torch.cuda.current_stream()
        if cur != self.stream:
            self.stream.wait_stream(cur)

    def publish(self):
        cur = torch.cuda.current_stream()
        if cur != self.stream:
            cur.wait_stream(self.stream)

    def set_state(self, st, history=None):
        self.wait_inputs()
        lmvd_set_state(self.h, st["z"], st["om"], st["m2"], st["mm1"], st["mm3"], history)

    def get_state(self, out=None, history=None):
        out = self.empty_state() if out is None else out
        self.wait_inputs()
        lmvd_get_state(self.h, out["z"], out["om"], out["m2"], out["mm1"], out["mm3"], history)
        self.publish()
        return out

    def history_buffer(self, device=None):
        dev = self.device if device is None else torch.device(device)
        return torch.zeros(lmvd_history_bytes(self.h), dtype=torch.uint8, device=dev)

    def field(self, which):
        nbytes = lmvd_field_bytes(self.h, which)
        if which == LMVD_FIELD_R_MEANS:
            out = torch.zeros(nbytes // 8, dtype=torch.float64, device=self.device)
        else:
            rows = nbytes // (16 * self.cfg.nz * (self.cfg.nx // 2 + 1))
            out = torch.zeros((rows, self.cfg.nz, self.cfg.nx // 2 + 1), dtype=torch.complex128, device=self.device)
        self.wait_inputs()
        lmvd_get_field(self.h, which, out)
        self.publish()
        return out

    def advance_substage(self):
        lmvd_advance_substage(self.h)

    def step(self, n):
        lmvd_step(self.h, n)

    def synchronize(self):
        lmvd_synchronize(self.h)

    def close(self):
        if self.h is not None:
            lmvd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
