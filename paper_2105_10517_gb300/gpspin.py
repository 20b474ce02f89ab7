"""Python binding of libgpspin (include/gpspin.h): argument marshalling only.

Every step of the split-step Crank-Nicolson method runs in the CUDA library;
this module builds it in-tree for sm_103a, loads it with ctypes and converts
numpy arrays and parameter dicts.  There is no CPU fallback: if the library is
missing or fails to load, every entry point raises.
"""
import ctypes
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB_PATH = os.path.join(PKG, "libgpspin.so")
BUILD_DIR = os.path.join(PKG, "_build")
SOURCES = ["gp_capi.cu", "gp_sweeps.cu", "gp_reduce.cu", "gp_noalloc.cu", "gp_batch.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-O3"]

IMAG, REAL = 0, 1
SPLIT_LIE, SPLIT_STRANG = 0, 1
DEBUG_POISON = 1
SO_NONE, SO_RASHBA, SO_DRESSELHAUS = 0, 1, 2
FP64, FP32_MIXED = 0, 1
SUB_P, SUB_X, SUB_Y = 0, 1, 2

STATUS = {0: "GP_OK", 1: "GP_ERR_ARG", 2: "GP_ERR_OOM", 3: "GP_ERR_CUDA", 4: "GP_ERR_NONFINITE",
          5: "GP_ERR_UNSUPPORTED", 6: "GP_ERR_TOO_LARGE", 7: "GP_ERR_TIMEOUT", 8: "GP_ERR_QUEUE_FULL"}

# Every symbol the public header declares (checked by the CPU tests).
EXPORTS = ["gp_create", "gp_destroy", "gp_set_params", "gp_set_state", "gp_get_state", "gp_init_gaussian",
           "gp_init_winding", "gp_set_magnetization", "gp_set_splitting", "gp_propagate", "gp_propagate_host", "gp_refine_fp64", "gp_observables", "gp_apply_substep", "gp_profile_step", "gp_autotune",
           "gp_tiling_info", "gp_set_tiling", "gp_set_debug", "gp_plan_tiling", "gp_check_wait_timeout",
           "gp_propagate_noalloc", "gp_request_bytes", "gp_batch_create", "gp_batch_destroy", "gp_batch_submit",
           "gp_batch_step", "gp_batch_poll", "gp_batch_use_graphs", "gp_batch_set_persistent", "gp_batch_set_running_limit",
           "gp_batch_set_queue_limit", "gp_batch_cancel", "gp_batch_error",
           "gp_inject_alloc_failure", "gp_checkpoint_bytes", "gp_checkpoint_save", "gp_checkpoint_load",
           "gp_strerror"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(lib, deps):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    """Compile the CUDA sources (in parallel, one -gencode for sm_103a) and link
    libgpspin.so next to this file.  Returns the library path."""
    deps = [os.path.join(CSRC, s) for s in SOURCES] + [os.path.join(CSRC, "gp_internal.cuh"),
                                                        os.path.join(CSRC, "gp_handle.cuh"),
                                                        os.path.join(ROOT, "include", "gpspin.h")]
    if not force and not _stale(LIB_PATH, deps):
        return LIB_PATH
    os.makedirs(BUILD_DIR, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD_DIR, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc] + NVCC_FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB_PATH + ".tmp"
    r = subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("xlen", ctypes.c_double), ("ylen", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("wx", ctypes.c_double), ("wy", ctypes.c_double),
        ("c0", ctypes.c_double), ("c2", ctypes.c_double), ("omeg", ctypes.c_double),
        ("so_type", ctypes.c_int),
        ("gamma", ctypes.c_double), ("rabi", ctypes.c_double),
        ("precision", ctypes.c_int),
    ]


class Obs(ctypes.Structure):
    _fields_ = [
        ("norm", ctypes.c_double * 3),
        ("norm_total", ctypes.c_double),
        ("magnetization", ctypes.c_double),
        ("energy", ctypes.c_double),
        ("mu", ctypes.c_double),
        ("steps", ctypes.c_longlong),
    ]


class Request(ctypes.Structure):
    _fields_ = [
        ("frac", ctypes.c_double * 3),
        ("seed", ctypes.c_ulonglong),
        ("phase_noise", ctypes.c_double),
        ("tol", ctypes.c_double),
        ("tol32", ctypes.c_double),
        ("cap", ctypes.c_longlong),
        ("policy", ctypes.c_int),
        ("refine_steps", ctypes.c_longlong),
    ]


POLICY_FP64, POLICY_FP32_REFINE = 0, 1
REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED, REQ_UNKNOWN, REQ_CANCELLED = 0, 1, 2, 3, 4, 5

_lib = None


def load():
    """Load libgpspin.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_2105_10517_gb300.gpspin.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    lib.gp_create.argtypes = [ctypes.POINTER(Params), vp, ctypes.POINTER(vp)]
    lib.gp_destroy.argtypes = [vp]
    lib.gp_destroy.restype = None
    lib.gp_set_params.argtypes = [vp, ctypes.POINTER(Params)]
    lib.gp_set_state.argtypes = [vp, dp, ip]
    lib.gp_get_state.argtypes = [vp, dp]
    lib.gp_init_gaussian.argtypes = [vp, dp, ctypes.c_ulonglong, ctypes.c_double]
    lib.gp_init_winding.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_int), ctypes.c_ulonglong, ctypes.c_double]
    lib.gp_init_winding.restype = ctypes.c_int
    lib.gp_set_splitting.argtypes = [vp, ip]
    lib.gp_set_splitting.restype = ctypes.c_int
    lib.gp_set_magnetization.argtypes = [vp, ip, ctypes.c_double]
    lib.gp_set_magnetization.restype = ctypes.c_int
    lib.gp_propagate.argtypes = [vp, ctypes.c_longlong, ip]
    lib.gp_propagate_host.argtypes = [vp, dp, ctypes.c_longlong, ip, dp]
    lib.gp_refine_fp64.argtypes = [vp, ctypes.c_longlong, ip]
    lib.gp_observables.argtypes = [vp, ctypes.POINTER(Obs)]
    lib.gp_apply_substep.argtypes = [vp, ip, ip]
    lib.gp_profile_step.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_float)]
    lib.gp_autotune.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_double)]
    lib.gp_autotune.restype = ctypes.c_int
    lib.gp_tiling_info.argtypes = [vp, ip, ip, ctypes.POINTER(ctypes.c_int)]
    lib.gp_tiling_info.restype = ctypes.c_int
    lib.gp_set_tiling.argtypes = [vp, ip, ip, ip, ip, ip, ip]
    lib.gp_set_debug.argtypes = [vp, ip]
    lib.gp_set_debug.restype = ctypes.c_int
    lib.gp_plan_tiling.argtypes = [ctypes.POINTER(Params), ip, ip, ctypes.POINTER(ctypes.c_int)]
    lib.gp_plan_tiling.restype = ctypes.c_int
    lib.gp_set_tiling.restype = ctypes.c_int
    lib.gp_check_wait_timeout.argtypes = [vp, ip]
    lib.gp_check_wait_timeout.restype = ctypes.c_int
    lib.gp_propagate_noalloc.argtypes = [ctypes.POINTER(Params), vp, ctypes.c_longlong, ip, vp]
    lib.gp_propagate_noalloc.restype = ctypes.c_int
    lib.gp_request_bytes.argtypes = [ctypes.POINTER(Params), ip]
    lib.gp_request_bytes.restype = ctypes.c_size_t
    lib.gp_batch_create.argtypes = [ctypes.c_size_t, ip, vp, ctypes.POINTER(vp)]
    lib.gp_batch_destroy.argtypes = [vp]
    lib.gp_batch_destroy.restype = None
    lib.gp_batch_submit.argtypes = [vp, ctypes.POINTER(Params), ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_longlong)]
    lib.gp_batch_step.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.gp_batch_poll.argtypes = [vp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong),
                                  ctypes.POINTER(Obs), dp, ip]
    lib.gp_batch_set_queue_limit.argtypes = [vp, ip]
    lib.gp_batch_use_graphs.argtypes = [vp, ip]
    lib.gp_batch_set_persistent.argtypes = [vp, ip]
    lib.gp_batch_set_running_limit.argtypes = [vp, ctypes.c_longlong]
    lib.gp_batch_set_running_limit.restype = ctypes.c_int
    lib.gp_batch_cancel.argtypes = [vp, ctypes.c_longlong]
    lib.gp_batch_error.argtypes = [vp, ctypes.c_longlong]
    for name in ("gp_batch_create", "gp_batch_submit", "gp_batch_step", "gp_batch_poll", "gp_batch_use_graphs",
                 "gp_batch_set_persistent", "gp_batch_set_running_limit", "gp_batch_set_queue_limit",
                 "gp_batch_cancel", "gp_batch_error"):
        getattr(lib, name).restype = ctypes.c_int
    lib.gp_inject_alloc_failure.argtypes = [ctypes.c_longlong]
    lib.gp_inject_alloc_failure.restype = None
    lib.gp_checkpoint_bytes.argtypes = [vp]
    lib.gp_checkpoint_bytes.restype = ctypes.c_size_t
    lib.gp_checkpoint_save.argtypes = [vp, vp, ctypes.c_size_t]
    lib.gp_checkpoint_save.restype = ctypes.c_int
    lib.gp_checkpoint_load.argtypes = [vp, vp, ctypes.c_size_t]
    lib.gp_checkpoint_load.restype = ctypes.c_int
    lib.gp_strerror.argtypes = [ip]
    lib.gp_strerror.restype = ctypes.c_char_p
    for name in ("gp_create", "gp_set_params", "gp_set_state", "gp_get_state", "gp_init_gaussian",
                 "gp_propagate", "gp_refine_fp64", "gp_observables", "gp_apply_substep", "gp_profile_step"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


class GPError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        msg = load().gp_strerror(status).decode()
        super().__init__(f"{what}: {STATUS.get(status, status)} ({msg})")


def _check(st, what):
    if st != 0:
        raise GPError(st, what)


PARAM_DEFAULTS = dict(wx=1.0, wy=1.0, c0=0.0, c2=0.0, omeg=0.0, so_type=0, gamma=0.0, rabi=0.0, precision=FP64)


def make_params(p):
    q = dict(PARAM_DEFAULTS)
    q.update({k: v for k, v in p.items() if k in Params.__dict__ or k in dict(Params._fields_)})
    return Params(int(q["nx"]), int(q["ny"]), float(q["xlen"]), float(q["ylen"]), float(q["dt"]),
                  float(q["wx"]), float(q["wy"]), float(q["c0"]), float(q["c2"]), float(q["omeg"]),
                  int(q["so_type"]), float(q["gamma"]), float(q["rabi"]), int(q["precision"]))


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def propagate_noalloc(params, psi_dev_ptr, nsteps, mode=IMAG, stream=None):
    """gp_propagate_noalloc on a caller-owned device buffer (an integer device
    address of psi[3][ny][nx] complex128, e.g. a torch tensor's data_ptr())."""
    p = make_params(params)
    s = ctypes.c_void_p(int(stream)) if stream is not None else None
    _check(load().gp_propagate_noalloc(ctypes.byref(p), ctypes.c_void_p(int(psi_dev_ptr)), int(nsteps), int(mode), s),
           "gp_propagate_noalloc")


def inject_alloc_failure(after):
    """Make the after-th device allocation of the library from now on fail once
    (0: the next one); after < 0 disarms (tests of out-of-memory handling)."""
    load().gp_inject_alloc_failure(int(after))


def plan_tiling(params, mode=IMAG):
    """Default tilings of the x- and y-pass for these parameters, computed on the
    host (no device needed)."""
    p = make_params(params)
    out = {}
    for d, name in ((0, "xpass"), (1, "ypass")):
        v = (ctypes.c_int * 12)()
        _check(load().gp_plan_tiling(ctypes.byref(p), int(mode), d, v), "gp_plan_tiling")
        out[name] = dict(cluster=v[0], lines_per_cta=v[1], chunk=v[2], chunks=v[3], threads=v[4], smem=v[5],
                         ctas=v[6], register_solve=bool(v[7]), fixup=v[8], chunk_stride=v[9], line_stride=v[10],
                         bank_conflicts=v[11])
    return out


class Solver:
    """One GP instance on the current CUDA device (a gp_handle)."""

    def __init__(self, params, stream=None):
        lib = load()
        self.params = dict(params)
        self._p = make_params(params)
        h = ctypes.c_void_p()
        s = ctypes.c_void_p(int(stream)) if stream is not None else None
        _check(lib.gp_create(ctypes.byref(self._p), s, ctypes.byref(h)), "gp_create")
        self._h = h
        self.nx, self.ny = self._p.nx, self._p.ny

    def close(self):
        if getattr(self, "_h", None):
            load().gp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_params(self, params):
        p = make_params(params)
        _check(load().gp_set_params(self._h, ctypes.byref(p)), "gp_set_params")
        self.params = dict(params)
        self._p = p

    def _host_ptr(self, buf, what):
        """Pointer to a host complex128 buffer of shape (3, ny, nx): a numpy array
        or a (pinned) torch CPU tensor."""
        if hasattr(buf, "data_ptr"):
            if tuple(buf.shape) != (3, self.ny, self.nx) or not buf.is_contiguous() or buf.is_cuda:
                raise ValueError(f"{what}: need a contiguous CPU tensor of shape (3, {self.ny}, {self.nx})")
            if str(buf.dtype) != "torch.complex128":
                raise ValueError(f"{what}: need complex128")
            return ctypes.cast(ctypes.c_void_p(buf.data_ptr()), ctypes.POINTER(ctypes.c_double)), buf
        a = np.ascontiguousarray(buf, dtype=np.complex128)
        if a.shape != (3, self.ny, self.nx):
            raise ValueError(f"{what}: psi must have shape (3, {self.ny}, {self.nx})")
        return _dptr(a), a

    def set_state(self, psi, normalize=False):
        ptr, keep = self._host_ptr(psi, "set_state")
        _check(load().gp_set_state(self._h, ptr, int(bool(normalize))), "gp_set_state")

    def get_state(self, out=None):
        if out is None:
            out = np.empty((3, self.ny, self.nx), dtype=np.complex128)
        elif not hasattr(out, "data_ptr") and (not isinstance(out, np.ndarray) or out.dtype != np.complex128
                                               or not out.flags.c_contiguous):
            raise ValueError("get_state: out must be a C-contiguous complex128 array")
        ptr, keep = self._host_ptr(out, "get_state")
        _check(load().gp_get_state(self._h, ptr), "gp_get_state")
        return out

    def propagate_host(self, psi_in, nsteps, mode=IMAG, out=None):
        """set_state(psi_in) + propagate(nsteps, mode) + get_state(out) in one
        library call (the first pass reads psi_in directly where the device can)."""
        if out is None:
            out = np.empty((3, self.ny, self.nx), dtype=np.complex128)
        elif not hasattr(out, "data_ptr") and (not isinstance(out, np.ndarray) or out.dtype != np.complex128
                                               or not out.flags.c_contiguous):
            raise ValueError("propagate_host: out must be a C-contiguous complex128 array")
        pin, keep_in = self._host_ptr(psi_in, "propagate_host")
        pout, keep_out = self._host_ptr(out, "propagate_host")
        _check(load().gp_propagate_host(self._h, pin, int(nsteps), int(mode), pout), "gp_propagate_host")
        return out

    def init_gaussian(self, frac=(0.25, 0.5, 0.25), seed=1, phase_noise=1e-3):
        f = np.asarray(frac, dtype=np.float64)
        _check(load().gp_init_gaussian(self._h, _dptr(f), int(seed), float(phase_noise)), "gp_init_gaussian")

    def init_winding(self, frac=(0.25, 0.5, 0.25), winding=(0, 0, 0), seed=1, phase_noise=1e-3):
        f = np.asarray(frac, dtype=np.float64)
        w = (ctypes.c_int * 3)(*[int(v) for v in winding])
        _check(load().gp_init_winding(self._h, _dptr(f), w, int(seed), float(phase_noise)), "gp_init_winding")

    def set_splitting(self, split):
        """SPLIT_LIE (default) or SPLIT_STRANG (second order, complex128 handles)."""
        _check(load().gp_set_splitting(self._h, int(split)), "gp_set_splitting")

    def set_magnetization(self, m):
        """Keep N = 1 and N+ - N- = m in imaginary time (None: plain renormalisation)."""
        _check(load().gp_set_magnetization(self._h, 0 if m is None else 1, 0.0 if m is None else float(m)),
               "gp_set_magnetization")

    def propagate(self, nsteps, mode=IMAG):
        _check(load().gp_propagate(self._h, int(nsteps), int(mode)), "gp_propagate")

    def refine_fp64(self, nsteps, mode=IMAG):
        """Widen an FP32-storage handle to FP64 and continue nsteps steps in FP64."""
        _check(load().gp_refine_fp64(self._h, int(nsteps), int(mode)), "gp_refine_fp64")

    def apply_substep(self, which, mode=IMAG):
        w = {"P": SUB_P, "X": SUB_X, "Y": SUB_Y}.get(which, which)
        _check(load().gp_apply_substep(self._h, int(w), int(mode)), "gp_apply_substep")

    def profile_step(self, mode=IMAG):
        """One step with per-kernel device times (ms): x-pass, y-pass, normalisation, whole step."""
        ms = (ctypes.c_float * 4)()
        _check(load().gp_profile_step(self._h, int(mode), ms), "gp_profile_step")
        return list(ms)

    def autotune(self, mode=IMAG):
        """Pick the fastest tiling of both line passes (state unchanged); returns their ms."""
        ms = ctypes.c_double()
        _check(load().gp_autotune(self._h, int(mode), ctypes.byref(ms)), "gp_autotune")
        return ms.value

    def set_debug(self, poison=True):
        """Poison check: every byte a pass must write is set to a NaN pattern first, so a
        skipped write shows up as a non-finite state (gp_set_debug, GP_DEBUG_POISON)."""
        _check(load().gp_set_debug(self._h, DEBUG_POISON if poison else 0), "gp_set_debug")

    def set_tiling(self, dir, cluster=1, lines_per_cta=1, chunk=0, mode=IMAG, register_solve=None):
        """Force the tiling of the x-pass (dir 0) or y-pass (dir 1); register_solve True / False
        selects the register-resident or shared-memory solve, None the precision's default."""
        rs = -1 if register_solve is None else int(bool(register_solve))
        _check(load().gp_set_tiling(self._h, int(mode), int(dir), int(cluster), int(lines_per_cta), int(chunk), rs),
               "gp_set_tiling")

    def tiling(self, mode=IMAG):
        """Tiling of the x- and y-pass: dicts of cluster size, lines per CTA, chunk length..."""
        out = {}
        for d, name in ((0, "xpass"), (1, "ypass")):
            v = (ctypes.c_int * 8)()
            _check(load().gp_tiling_info(self._h, int(mode), d, v), "gp_tiling_info")
            out[name] = dict(cluster=v[0], lines_per_cta=v[1], chunk=v[2], chunks=v[3], threads=v[4], smem=v[5],
                             ctas=v[6], register_solve=bool(v[7]))
        return out

    def checkpoint(self):
        """The handle's exact state as bytes (gp_checkpoint_save)."""
        n = int(load().gp_checkpoint_bytes(self._h))
        buf = ctypes.create_string_buffer(n)
        _check(load().gp_checkpoint_save(self._h, ctypes.cast(buf, ctypes.c_void_p), n), "gp_checkpoint_save")
        return buf.raw

    def restore(self, data):
        """Restore a checkpoint made by checkpoint() (same grid and precision)."""
        buf = ctypes.create_string_buffer(bytes(data), len(data))
        _check(load().gp_checkpoint_load(self._h, ctypes.cast(buf, ctypes.c_void_p), len(data)),
               "gp_checkpoint_load")

    def save_checkpoint(self, path):
        with open(path, "wb") as f:
            f.write(self.checkpoint())

    def load_checkpoint(self, path):
        with open(path, "rb") as f:
            self.restore(f.read())

    def check_wait_timeout(self, polls=64):
        """Run the passes' bounded device wait on a barrier nothing completes
        (raises GPError with GP_ERR_TIMEOUT, as a propagate whose copy wait gave up)."""
        _check(load().gp_check_wait_timeout(self._h, int(polls)), "gp_check_wait_timeout")

    def observables(self):
        o = Obs()
        _check(load().gp_observables(self._h, ctypes.byref(o)), "gp_observables")
        return dict(norm=np.array(o.norm[:]), norm_total=o.norm_total, magnetization=o.magnetization,
                    energy=o.energy, mu=o.mu, steps=o.steps)


def request_bytes(params, policy=POLICY_FP64):
    return int(load().gp_request_bytes(ctypes.byref(make_params(params)), int(policy)))


class Batch:
    """A gp_batch: continuously batched imaginary-time solves on the current device."""

    def __init__(self, max_bytes, check_every=100, stream=None):
        lib = load()
        b = ctypes.c_void_p()
        s = ctypes.c_void_p(int(stream)) if stream is not None else None
        _check(lib.gp_batch_create(ctypes.c_size_t(int(max_bytes)), int(check_every), s, ctypes.byref(b)),
               "gp_batch_create")
        self._b = b
        self.check_every = check_every
        self._shape = {}

    def close(self):
        if getattr(self, "_b", None):
            load().gp_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, params, frac=(0.25, 0.5, 0.25), seed=1, phase_noise=1e-3, tol=1e-9, tol32=1e-7, cap=20000,
               policy=POLICY_FP64, refine_steps=2000):
        r = Request((ctypes.c_double * 3)(*frac), int(seed), float(phase_noise), float(tol), float(tol32), int(cap),
                    int(policy), int(refine_steps))
        rid = ctypes.c_longlong()
        _check(load().gp_batch_submit(self._b, ctypes.byref(make_params(params)), ctypes.byref(r), ctypes.byref(rid)),
               "gp_batch_submit")
        self._shape[rid.value] = (3, int(params["ny"]), int(params["nx"]))
        return rid.value

    def use_graphs(self, enable=True):
        """Replay captured ticks while the running set is unchanged (default) or launch directly."""
        _check(load().gp_batch_use_graphs(self._b, int(bool(enable))), "gp_batch_use_graphs")

    def set_persistent(self, max_ctas=0):
        """Batched launch form: 0 persistent, one CTA per resident slot, CTAs taking the work items
        from a counter; > 0 the same with at most max_ctas CTAs; None or < 0 one CTA per work item
        (the batch's default)."""
        v = -1 if max_ctas is None else int(max_ctas)
        _check(load().gp_batch_set_persistent(self._b, v), "gp_batch_set_persistent")

    def set_running_limit(self, max_sites):
        """Admit while the running solves' grid points stay within max_sites (0: no limit)."""
        _check(load().gp_batch_set_running_limit(self._b, int(max_sites)), "gp_batch_set_running_limit")

    def set_queue_limit(self, max_queued):
        """Refuse submissions (GP_ERR_QUEUE_FULL) while max_queued requests wait; 0: no limit."""
        _check(load().gp_batch_set_queue_limit(self._b, int(max_queued)), "gp_batch_set_queue_limit")

    def cancel(self, rid):
        """Cancel a queued or running solve (its device memory is released at once)."""
        _check(load().gp_batch_cancel(self._b, int(rid)), "gp_batch_cancel")

    def error(self, rid):
        """The status that failed a REQ_FAILED solve (0 otherwise)."""
        return int(load().gp_batch_error(self._b, int(rid)))

    def step(self):
        nr, nq = ctypes.c_int(), ctypes.c_int()
        _check(load().gp_batch_step(self._b, ctypes.byref(nr), ctypes.byref(nq)), "gp_batch_step")
        return nr.value, nq.value

    def poll(self, rid, fetch=False, release=False):
        """(state, steps, observables dict, psi or None)."""
        st, steps, o = ctypes.c_int(), ctypes.c_longlong(), Obs()
        psi = np.empty(self._shape[rid], dtype=np.complex128) if fetch else None
        ptr = _dptr(psi) if fetch else None
        _check(load().gp_batch_poll(self._b, int(rid), ctypes.byref(st), ctypes.byref(steps), ctypes.byref(o), ptr,
                                    int(bool(release))), "gp_batch_poll")
        obs = dict(norm=np.array(o.norm[:]), norm_total=o.norm_total, magnetization=o.magnetization,
                   energy=o.energy, mu=o.mu, steps=o.steps)
        if fetch and st.value != REQ_DONE:
            psi = None
        return st.value, steps.value, obs, psi
