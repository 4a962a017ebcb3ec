"""GB300 collisional-PIC step for XFEL-heated solid Al (Royle et al., PICLS).

Thin Python binding of the C ABI in include/pic.h: argument marshalling
only.  Every step of the simulation runs in the CUDA kernels of
paper_1704_01202_gb300/csrc, compiled for sm_103a into
paper_1704_01202_gb300/_build/libpicgb.so (FP32 state and arithmetic) and,
from the same sources, libpicgb64.so (the same kernels in FP64, used to
check the device logic against the FP64 oracle without single-precision
rounding).  There is no CPU path: if the library or a GPU is missing, the
calls raise.

PyTorch provides the device memory (one uint8 arena tensor per context)
and the CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc")
_BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_BUILD, "libpicgb.so")
LIB64_PATH = os.path.join(_BUILD, "libpicgb64.so")
_INCLUDE = os.path.join(os.path.dirname(_HERE), "include")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

_lock = threading.Lock()
_lib = None
_lib64 = None

NSUB, NZ, MAX_BINS = 5, 14, 8
STATUS = {0: "PIC_OK", 1: "PIC_ERR_ARG", 2: "PIC_ERR_OOM", 3: "PIC_ERR_TABLE", 4: "PIC_ERR_CUDA",
          5: "PIC_ERR_TIMEOUT", 6: "PIC_ERR_NUMERIC", 7: "PIC_ERR_STATE", 8: "PIC_ERR_CAPACITY"}
COUNT_NAMES = ["ION", "ION_REJ", "REC", "PH0", "PH1", "PH2", "PH3", "PH4", "PART", "AUG", "KA",
               "PGT1", "ESC_E", "ESC_I", "EE", "EI"]
ABI_FUNCTIONS = ["pic_required_bytes", "pic_init", "pic_source", "pic_load_electrons", "pic_load_ions",
                 "pic_set_photons", "pic_set_fields", "pic_step", "pic_sync", "pic_diagnostics",
                 "pic_counts", "pic_get_electrons", "pic_get_ions", "pic_get_photons", "pic_get_fields",
                 "pic_get_current", "pic_launch_count", "pic_free", "pic_last_error", "pic_philox_check",
                 "pic_timing", "pic_batch_required_bytes", "pic_batch_init", "pic_batch_admit",
                 "pic_batch_retire", "pic_batch_set_budget", "pic_batch_slot", "pic_batch_diagnostics", "pic_batch_counts",
                 "pic_batch_get_electrons", "pic_batch_get_ions", "pic_philox_check_static",
                 "pic_use_graphs", "pic_autotune", "pic_order_check", "pic_dd_sum_check", "pic_seed", "pic_checkpoint_bytes", "pic_checkpoint", "pic_restore",
                 "pic_get_electrons64", "pic_get_ions64", "pic_real_bytes",
                 "pic_rt", "pic_rt_get", "pic_rt_set", "pic_rt_cells"]


def _sources():
    return sorted(os.path.join(_SRC, f) for f in os.listdir(_SRC) if f.endswith((".cu", ".cuh")))


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the CUDA library for sm_103a (nvcc cross-compiles without a
    GPU): the FP32 build and the FP64 build, in parallel.  Returns the FP32
    library's path."""
    srcs = _sources() + [os.path.join(_INCLUDE, "pic.h"), os.path.abspath(__file__)]
    newest = max(os.path.getmtime(s) for s in srcs)
    # FP32 build: approximate single-precision division and square root
    # (within 2-3 ulp) and denormals flushed to zero; the FP64 build's double
    # arithmetic is IEEE either way
    fast32 = ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"]
    todo = [(path, flags) for path, flags in ((LIB_PATH, fast32), (LIB64_PATH, ["-DPIC_FP64"]))
            if force or not os.path.exists(path) or os.path.getmtime(path) < newest]
    if not todo:
        return LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    procs = []
    for path, flags in todo:
        tmp = path + f".{os.getpid()}.tmp"
        cmd = ["nvcc", ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC,-pthread", *flags,
               "-o", tmp, os.path.join(_SRC, "pic_api.cu")]
        procs.append((path, tmp, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)))
    errors = []
    for path, tmp, pr in procs:
        _, err = pr.communicate()
        if pr.returncode != 0:
            errors.append(f"nvcc failed for {os.path.basename(path)}:\n" + err[-4000:])
            continue
        if verbose:
            print(err)
        os.replace(tmp, path)
    if errors:
        raise RuntimeError("\n".join(errors))
    return LIB_PATH


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("dx_nm", C.c_double), ("dy_nm", C.c_double),
                ("dt_fs", C.c_double), ("rad_every", C.c_int), ("seed", C.c_uint64), ("cfl", C.c_double)]


class Species(C.Structure):
    _fields_ = [("n_ref_cm3", C.c_double), ("w_ion", C.c_double), ("m_ion_me", C.c_double),
                ("E_bulk_eV", C.c_double), ("ipd_model", C.c_int), ("coulomb_log", C.c_double),
                ("flags", C.c_uint), ("cap_e", C.c_int), ("cap_i", C.c_int)]


class Tables(C.Structure):
    _fields_ = [("lotz_a", C.c_double * NSUB), ("lotz_b", C.c_double * NSUB), ("lotz_c", C.c_double * NSUB),
                ("E_bind", (C.c_double * NSUB) * NZ), ("tauK", (C.c_double * 2) * NZ),
                ("omegaK", (C.c_double * 2) * NZ), ("E_Kalpha", C.c_double * NZ),
                ("n_hv", C.c_int), ("hv_tab", C.POINTER(C.c_double)), ("sigma_photo", C.POINTER(C.c_double)),
                ("n_T", C.c_int), ("n_n", C.c_int), ("eos_T", C.POINTER(C.c_double)),
                ("eos_n", C.POINTER(C.c_double)), ("eos_Zbar", C.POINTER(C.c_double))]


class Pulse(C.Structure):
    _fields_ = [("shape", C.c_int), ("I_peak_Wcm2", C.c_double), ("fwhm_fs", C.c_double),
                ("t_peak_fs", C.c_double), ("hv_eV", C.c_double), ("bandwidth_eV", C.c_double),
                ("n_bins", C.c_int), ("spot_sigma_nm", C.c_double)]


class Diag(C.Structure):
    _fields_ = [("csd", C.POINTER(C.c_double)), ("eedf", C.POINTER(C.c_double)), ("n_E", C.c_int),
                ("E_max_eV", C.c_double), ("t_fs", C.c_double), ("transmission", C.c_double),
                ("T_e_eV", C.c_double), ("n_e_cm3", C.c_double), ("Zbar", C.c_double),
                ("ke_e", C.c_double), ("ke_i", C.c_double), ("e_ion", C.c_double), ("e_phot", C.c_double),
                ("e_inc", C.c_double), ("e_trans", C.c_double), ("e_ka_esc", C.c_double),
                ("e_esc", C.c_double), ("e_field", C.c_double), ("counts", C.c_uint64 * 16),
                ("n_e", C.c_int64), ("n_i", C.c_int64),
                ("e_back", C.c_double), ("e_rt_num", C.c_double), ("e_rt_pend", C.c_double)]


class SeedSpec(C.Structure):
    _fields_ = [("ppc_e", C.c_int), ("ppc_i", C.c_int), ("Z_init", C.c_int), ("T_e_eV", C.c_double),
                ("T_i_eV", C.c_double), ("beam_frac", C.c_double), ("beam_E_eV", C.c_double),
                ("seed", C.c_uint64)]


class RTConfig(C.Structure):
    _fields_ = [("coarsen", C.c_int), ("n_polar", C.c_int), ("n_azimuth", C.c_int), ("scheme", C.c_int)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_F = C.POINTER(C.c_float)


def lib(fp64: bool = False):
    """Load the compiled library, the FP32 build or (fp64) the FP64 build
    (raises if it has not been built)."""
    global _lib, _lib64
    with _lock:
        if (_lib64 if fp64 else _lib) is None:
            path = LIB64_PATH if fp64 else LIB_PATH
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library missing: {path} (run __graft_entry__.build())")
            L = C.CDLL(path)
            L.pic_required_bytes.restype = C.c_size_t
            L.pic_required_bytes.argtypes = [C.POINTER(Grid), C.POINTER(Species), C.c_int, C.c_int]
            L.pic_init.argtypes = [C.POINTER(_P), C.POINTER(Grid), C.POINTER(Species), C.POINTER(Tables),
                                   _P, C.c_size_t, _P]
            L.pic_source.argtypes = [_P, C.POINTER(Pulse)]
            L.pic_load_electrons.argtypes = [_P, C.c_int64, _D, _D, _F, _F, C.POINTER(C.c_uint64)]
            L.pic_load_ions.argtypes = [_P, C.c_int64, _D, _D, _F, _F, C.POINTER(C.c_int32),
                                        C.POINTER(C.c_int32), C.POINTER(C.c_uint32)]
            L.pic_set_photons.argtypes = [_P, _D]
            L.pic_set_fields.argtypes = [_P, _F]
            L.pic_step.argtypes = [_P, C.c_int]
            L.pic_sync.argtypes = [_P]
            L.pic_diagnostics.argtypes = [_P, C.POINTER(Diag)]
            L.pic_counts.argtypes = [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
            L.pic_get_electrons.argtypes = [_P, _D, _D, _F, _F, C.POINTER(C.c_uint64)]
            L.pic_get_ions.argtypes = [_P, _D, _D, _F, _F, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                       C.POINTER(C.c_uint32)]
            L.pic_get_electrons64.argtypes = [_P, _D, _D, _D, _D, C.POINTER(C.c_uint64)]
            L.pic_get_ions64.argtypes = [_P, _D, _D, _D, _D, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                         C.POINTER(C.c_uint32)]
            L.pic_get_photons.argtypes = [_P, _D]
            L.pic_get_fields.argtypes = [_P, _F]
            L.pic_get_current.argtypes = [_P, _D]
            L.pic_launch_count.restype = C.c_int64
            L.pic_launch_count.argtypes = [_P]
            L.pic_free.argtypes = [_P]
            L.pic_last_error.restype = C.c_char_p
            L.pic_last_error.argtypes = [_P]
            L.pic_philox_check.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                           C.POINTER(C.c_uint32), C.c_int]
            L.pic_philox_check_static.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                                  C.POINTER(C.c_uint32), C.c_int]
            L.pic_use_graphs.argtypes = [_P, C.c_int]
            L.pic_order_check.argtypes = [C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.c_int, C.c_int,
                                          C.POINTER(C.c_uint16)]
            L.pic_dd_sum_check.argtypes = [_F, C.c_int, _D]
            L.pic_seed.argtypes = [_P, C.POINTER(SeedSpec)]
            L.pic_checkpoint_bytes.argtypes = [_P]
            L.pic_checkpoint_bytes.restype = C.c_size_t
            L.pic_checkpoint.argtypes = [_P, C.c_void_p, C.c_size_t]
            L.pic_restore.argtypes = [_P, C.c_void_p, C.c_size_t]
            L.pic_autotune.argtypes = [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_float)]
            L.pic_timing.argtypes = [_P, C.c_int, _D, C.POINTER(C.c_int64)]
            L.pic_rt.argtypes = [_P, C.POINTER(RTConfig)]
            L.pic_rt_get.argtypes = [_P, _D, _D, _D]
            L.pic_rt_set.argtypes = [_P, _D, _D, _D]
            L.pic_rt_cells.argtypes = [_P, _D, _D, _D, _D]
            L.pic_batch_required_bytes.restype = C.c_size_t
            L.pic_batch_required_bytes.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int]
            L.pic_batch_init.argtypes = [C.POINTER(_P), C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(Tables),
                                         _P, C.c_size_t, _P]
            L.pic_batch_admit.argtypes = [_P, C.POINTER(Grid), C.POINTER(Species), C.POINTER(Pulse),
                                          C.c_int64, _D, _D, _F, _F, C.POINTER(C.c_uint64),
                                          C.c_int64, _D, _D, _F, _F, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                          C.POINTER(C.c_uint32), C.POINTER(C.c_int)]
            L.pic_batch_retire.argtypes = [_P, C.c_int]
            L.pic_batch_slot.argtypes = [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_uint32)]
            L.pic_batch_set_budget.argtypes = [_P, C.c_int, C.c_int64]
            L.pic_batch_diagnostics.argtypes = [_P, C.c_int, C.POINTER(Diag)]
            L.pic_batch_counts.argtypes = [_P, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
            L.pic_batch_get_electrons.argtypes = [_P, C.c_int, _D, _D, _F, _F, C.POINTER(C.c_uint64)]
            L.pic_batch_get_ions.argtypes = [_P, C.c_int, _D, _D, _F, _F, C.POINTER(C.c_int32),
                                             C.POINTER(C.c_int32), C.POINTER(C.c_uint32)]
            for name in ABI_FUNCTIONS:
                if name not in ("pic_required_bytes", "pic_launch_count", "pic_last_error",
                                "pic_batch_required_bytes", "pic_checkpoint_bytes"):
                    getattr(L, name).restype = C.c_int
            if L.pic_real_bytes() != (8 if fp64 else 4):
                raise RuntimeError(f"{path} is not the {'FP64' if fp64 else 'FP32'} build")
            if fp64:
                _lib64 = L
            else:
                _lib = L
    return _lib64 if fp64 else _lib


class PicError(RuntimeError):
    pass


def _p(a, t=C.c_double):
    return a.ctypes.data_as(C.POINTER(t))


def _tables(tab: dict):
    t = Tables()
    for s in range(NSUB):
        t.lotz_a[s] = float(tab["lotz_a"][s])
        t.lotz_b[s] = float(tab["lotz_b"][s])
        t.lotz_c[s] = float(tab["lotz_c"][s])
    for z in range(NZ):
        for s in range(NSUB):
            t.E_bind[z][s] = float(tab["E_bind"][z, s])
        for k in range(2):
            t.tauK[z][k] = float(tab["tauK"][z, k])
            t.omegaK[z][k] = float(tab["omegaK"][z, k])
        t.E_Kalpha[z] = float(tab["E_Kalpha"][z])
    keep = [np.ascontiguousarray(tab[k], dtype=np.float64)
            for k in ("hv_tab", "sigma_photo", "eos_T", "eos_n", "eos_Zbar")]
    t.n_hv = keep[0].size
    t.hv_tab, t.sigma_photo = _p(keep[0]), _p(keep[1])
    t.n_T, t.n_n = keep[2].size, keep[3].size
    t.eos_T, t.eos_n, t.eos_Zbar = _p(keep[2]), _p(keep[3]), _p(keep[4])
    return t, keep


def pulse_struct(pl) -> Pulse:
    return Pulse(shape=pl.shape, I_peak_Wcm2=pl.I_peak_Wcm2, fwhm_fs=pl.fwhm_fs, t_peak_fs=pl.t_peak_fs,
                 hv_eV=pl.hv_eV, bandwidth_eV=pl.bandwidth_eV, n_bins=pl.n_bins, spot_sigma_nm=pl.spot_sigma_nm)


def default_capacity(n_e: int, n_i: int, z_init: int, headroom: float = 1.3) -> tuple[int, int]:
    """Electron capacity for every ion fully stripped (plus headroom)."""
    cap_e = int((n_e + n_i * (13 - z_init)) * headroom) + 1024
    return cap_e, n_i + 1024


def check_capacity(cap_e: int, cap_i: int) -> None:
    """Refuse capacities the C ABI cannot take, before they reach a 32-bit
    ctypes field (which would wrap them silently): both positive and
    cap_e + 3 cap_i below 2^31 (a step appends at most three electrons per
    ion after the held ones, and particle indices are 32-bit)."""
    if cap_e <= 0 or cap_i <= 0 or cap_e + 3 * cap_i > (1 << 31) - 1:
        raise PicError(f"capacity cap_e={cap_e}, cap_i={cap_i} out of range: both > 0 and "
                       f"cap_e + 3 cap_i < 2^31; pass smaller capacities")


class Slab:
    """One slab on the GPU, driven through the C ABI."""

    def __init__(self, cfg, tables: dict, pulse=None, cap_e: int = 0, cap_i: int = 0,
                 use_torch_arena: bool = True, stream=None, fp64: bool = False):
        self.L = lib(fp64)
        self.cfg = cfg
        self.grid = _grid(cfg)
        if cap_e <= 0 or cap_i <= 0:
            ce, ci = default_capacity(cfg.ncell * cfg.ppc_e, cfg.ncell * cfg.ppc_i, cfg.Z_init)
            cap_e = cap_e if cap_e > 0 else ce
            cap_i = cap_i if cap_i > 0 else ci
        check_capacity(cap_e, cap_i)
        self.species = _species(cfg, cap_e, cap_i)
        self._t, self._keep = _tables(tables)
        self.arena = None
        arena_ptr, arena_bytes = None, 0
        stream_ptr = None
        if use_torch_arena:
            import torch
            if not torch.cuda.is_available():
                raise PicError("no CUDA device")
            nbytes = self.L.pic_required_bytes(C.byref(self.grid), C.byref(self.species), 0, 0)
            self.arena = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            arena_ptr, arena_bytes = self.arena.data_ptr(), nbytes
            s = stream if stream is not None else torch.cuda.current_stream()
            stream_ptr = s.cuda_stream
        self.h = C.c_void_p()
        st = self.L.pic_init(C.byref(self.h), C.byref(self.grid), C.byref(self.species), C.byref(self._t),
                             arena_ptr, arena_bytes, stream_ptr)
        if st != 0:
            raise PicError(f"pic_init: {STATUS.get(st, st)}")
        self.n_bins = 0
        if pulse is not None:
            self.set_pulse(pulse)

    def _check(self, st, what):
        if st != 0:
            msg = self.L.pic_last_error(self.h).decode() if self.h else ""
            raise PicError(f"{what}: {STATUS.get(st, st)} {msg}")

    def close(self):
        if getattr(self, "h", None):
            self.L.pic_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_pulse(self, pl):
        self._check(self.L.pic_source(self.h, C.byref(pulse_struct(pl))), "pic_source")
        self.n_bins = pl.n_bins

    def set_rt(self, coarsen=5, n_polar=4, n_azimuth=2, scheme=0):
        """Radiation transport instead of the ballistic march (pic_rt)."""
        r = RTConfig(coarsen=coarsen, n_polar=n_polar, n_azimuth=n_azimuth, scheme=scheme)
        self._check(self.L.pic_rt(self.h, C.byref(r)), "pic_rt")
        self.rt = r
        self.nrx = self.cfg.nx // coarsen
        self.nry = self.cfg.ny // coarsen if self.cfg.ny > 1 else 1
        self.nord = 1 + n_polar * (n_azimuth if self.cfg.ny > 1 else 1)

    def rt_field(self):
        shp = (self.nord, self.n_bins, self.nry, self.nrx)
        F, Gx, Gy = np.zeros(shp), np.zeros(shp), np.zeros(shp)
        self._check(self.L.pic_rt_get(self.h, _p(F), _p(Gx), _p(Gy)), "pic_rt_get")
        return F, Gx, Gy

    def set_rt_field(self, F, Gx=None, Gy=None):
        F = np.ascontiguousarray(F, dtype=np.float64)
        Gx = np.zeros_like(F) if Gx is None else np.ascontiguousarray(Gx, dtype=np.float64)
        Gy = np.zeros_like(F) if Gy is None else np.ascontiguousarray(Gy, dtype=np.float64)
        n = self.nord * self.n_bins * self.nry * self.nrx
        for name, x in (("F", F), ("Gx", Gx), ("Gy", Gy)):
            _expect_size(x, n, f"rad field {name}")
        self._check(self.L.pic_rt_set(self.h, _p(F), _p(Gx), _p(Gy)), "pic_rt_set")

    def rt_cells(self):
        nc = self.cfg.nx * self.cfg.ny
        chi, emc, w, dE = np.zeros((nc, self.n_bins)), np.zeros(nc), np.zeros(nc), np.zeros(nc)
        self._check(self.L.pic_rt_cells(self.h, _p(chi), _p(emc), _p(w), _p(dE)), "pic_rt_cells")
        return dict(chi=chi, emc=emc, w=w, dE=dE)

    def load(self, st):
        _ek, e = _electron_args(st)
        self._check(self.L.pic_load_electrons(self.h, *e), "pic_load_electrons")
        _ik, i = _ion_args(st)
        self._check(self.L.pic_load_ions(self.h, *i), "pic_load_ions")

    def seed(self, seed=None):
        """Seed the initial plasma of the slab's configuration on the device
        (pic_seed): ppc, temperatures, beam and Z_init of the config; the
        config's seed unless one is given."""
        c = self.cfg
        spec = SeedSpec(c.ppc_e, c.ppc_i, c.Z_init, c.T_e_eV, c.T_i_eV, c.beam_frac, c.beam_E_eV,
                        int(c.seed if seed is None else seed))
        self._check(self.L.pic_seed(self.h, C.byref(spec)), "pic_seed")

    def checkpoint(self) -> bytes:
        """Host image of the slab's state (pic_checkpoint)."""
        n = self.L.pic_checkpoint_bytes(self.h)
        if n == 0:
            raise PicError("pic_checkpoint_bytes: nothing to checkpoint")
        buf = C.create_string_buffer(n)
        self._check(self.L.pic_checkpoint(self.h, buf, n), "pic_checkpoint")
        return buf.raw

    def restore(self, image: bytes):
        """Load a host image written by checkpoint() (pic_restore)."""
        buf = C.create_string_buffer(image, len(image))
        self._check(self.L.pic_restore(self.h, buf, len(image)), "pic_restore")

    def step(self, n=1):
        self._check(self.L.pic_step(self.h, n), "pic_step")

    def sync(self):
        self._check(self.L.pic_sync(self.h), "pic_sync")

    @property
    def launches(self):
        return self.L.pic_launch_count(self.h)

    def use_graphs(self, enable: bool):
        self._check(self.L.pic_use_graphs(self.h, 1 if enable else 0), "pic_use_graphs")

    def autotune(self, enable=None):
        """Switch the launch-shape autotuner on / off (None: leave it); returns
        the warps per CTA in use and the step times measured for 1, 2, 4, 8."""
        w = C.c_int()
        ms = np.zeros(4, dtype=np.float32)
        e = -1 if enable is None else (1 if enable else 0)
        self._check(self.L.pic_autotune(self.h, e, C.byref(w), _p(ms, C.c_float)), "pic_autotune")
        return w.value, ms

    def timing(self, enable=None):
        """Start (True) / stop (False) event timing; with None return the
        summed device times {cell, march, push, sort, field, step} (ms) and
        the number of recorded steps."""
        if enable is not None:
            self._check(self.L.pic_timing(self.h, 1 if enable else 0, None, None), "pic_timing")
            return None
        out = np.zeros(6)
        n = C.c_int64()
        self._check(self.L.pic_timing(self.h, -1, _p(out), C.byref(n)), "pic_timing")
        return dict(zip(("cell", "march", "push", "sort", "field", "step"), out)), n.value

    def counts(self):
        ne, ni = C.c_int64(), C.c_int64()
        self._check(self.L.pic_counts(self.h, C.byref(ne), C.byref(ni)), "pic_counts")
        return ne.value, ni.value

    def electrons(self, full: bool = False):
        """Electrons on the host; full: momenta and weights in double
        precision (the FP64 build's state as it is)."""
        n, _ = self.counts()
        d, args = _electron_out(n, full)
        f = self.L.pic_get_electrons64 if full else self.L.pic_get_electrons
        self._check(f(self.h, *args), "pic_get_electrons")
        return d

    def ions(self, full: bool = False):
        _, n = self.counts()
        d, args = _ion_out(n, full)
        f = self.L.pic_get_ions64 if full else self.L.pic_get_ions
        self._check(f(self.h, *args), "pic_get_ions")
        return d

    def set_photons(self, ph):
        a = np.ascontiguousarray(ph, dtype=np.float64)
        _expect_size(a, self.cfg.ny * self.cfg.nx * self.n_bins, "photon numbers")
        self._check(self.L.pic_set_photons(self.h, _p(a)), "pic_set_photons")

    def photons(self):
        a = np.zeros((self.cfg.ny, self.cfg.nx, max(self.n_bins, 1)))
        self._check(self.L.pic_get_photons(self.h, _p(a)), "pic_get_photons")
        return a

    def set_fields(self, f: dict):
        a = np.ascontiguousarray(np.stack([f[k] for k in ("ex", "ey", "ez", "bx", "by", "bz")]), dtype=np.float32)
        _expect_size(a, 6 * self.cfg.ny * (self.cfg.nx + 1), "fields")
        self._check(self.L.pic_set_fields(self.h, _p(a, C.c_float)), "pic_set_fields")

    def fields(self):
        a = np.zeros((6, self.cfg.ny, self.cfg.nx + 1), dtype=np.float32)
        self._check(self.L.pic_get_fields(self.h, _p(a, C.c_float)), "pic_get_fields")
        return dict(zip(("ex", "ey", "ez", "bx", "by", "bz"), a))

    def current(self):
        a = np.zeros((3, self.cfg.ny, self.cfg.nx + 1))
        self._check(self.L.pic_get_current(self.h, _p(a)), "pic_get_current")
        return a

    def diagnostics(self, n_E=64, E_max=1e4):
        d, finish = _diag_out(n_E, E_max)
        self._check(self.L.pic_diagnostics(self.h, C.byref(d)), "pic_diagnostics")
        return finish()


def _expect_size(a, n, what):
    """The library reads n values: refuse an array of another size."""
    if a.size != n:
        raise PicError(f"{what}: {a.size} values where the slab has {n}")


def _same_length(kind, n, *arrays, u):
    """The library reads n of each: refuse arrays of another length (or a
    momentum array that is not n x 3) instead of reading past them."""
    if any(x.ndim != 1 or x.size != n for x in arrays) or u.shape != (n, 3):
        raise PicError(f"{kind} arrays of different lengths: {[x.shape for x in arrays]} and u {u.shape} "
                       f"for {n} particles")


def _electron_args(st):
    """Contiguous copies of a particle state's electrons and the (n, X, Y, u,
    w, id) arguments pointing into them (keep the copies alive for the call)."""
    a = [np.ascontiguousarray(st.eX, dtype=np.float64), np.ascontiguousarray(st.eY, dtype=np.float64),
         np.ascontiguousarray(st.eu, dtype=np.float32), np.ascontiguousarray(st.ew, dtype=np.float32),
         np.ascontiguousarray(st.eid, dtype=np.uint64)]
    _same_length("electron", a[0].size, a[1], a[3], a[4], u=a[2])
    return a, (a[0].size, _p(a[0]), _p(a[1]), _p(a[2], C.c_float), _p(a[3], C.c_float), _p(a[4], C.c_uint64))


def _ion_args(st):
    a = [np.ascontiguousarray(st.iX, dtype=np.float64), np.ascontiguousarray(st.iY, dtype=np.float64),
         np.ascontiguousarray(st.iu, dtype=np.float32), np.ascontiguousarray(st.izf, dtype=np.float32),
         np.ascontiguousarray(st.iZ, dtype=np.int32), np.ascontiguousarray(st.inK, dtype=np.int32),
         np.ascontiguousarray(st.iid, dtype=np.uint32)]
    _same_length("ion", a[0].size, a[1], a[3], a[4], a[5], a[6], u=a[2])
    return a, (a[0].size, _p(a[0]), _p(a[1]), _p(a[2], C.c_float), _p(a[3], C.c_float), _p(a[4], C.c_int32),
            _p(a[5], C.c_int32), _p(a[6], C.c_uint32))


def _electron_out(n, full=False):
    ft, ct = (np.float64, C.c_double) if full else (np.float32, C.c_float)
    d = dict(X=np.zeros(n), Y=np.zeros(n), u=np.zeros((n, 3), dtype=ft), w=np.zeros(n, dtype=ft),
             id=np.zeros(n, dtype=np.uint64))
    return d, (_p(d["X"]), _p(d["Y"]), _p(d["u"], ct), _p(d["w"], ct), _p(d["id"], C.c_uint64))


def _ion_out(n, full=False):
    ft, ct = (np.float64, C.c_double) if full else (np.float32, C.c_float)
    d = dict(X=np.zeros(n), Y=np.zeros(n), u=np.zeros((n, 3), dtype=ft), zf=np.zeros(n, dtype=ft),
             Z=np.zeros(n, dtype=np.int32), nK=np.zeros(n, dtype=np.int32), id=np.zeros(n, dtype=np.uint32))
    return d, (_p(d["X"]), _p(d["Y"]), _p(d["u"], ct), _p(d["zf"], ct), _p(d["Z"], C.c_int32),
               _p(d["nK"], C.c_int32), _p(d["id"], C.c_uint32))


def _diag_out(n_E, E_max):
    csd = np.zeros(NZ)
    eedf = np.zeros(n_E)
    d = Diag(csd=_p(csd), eedf=_p(eedf), n_E=n_E, E_max_eV=E_max)

    def finish():
        out = {k: getattr(d, k) for k, _ in Diag._fields_ if k not in ("csd", "eedf", "counts")}
        out["csd"] = csd
        out["eedf"] = eedf
        out["counts"] = dict(zip(COUNT_NAMES, (int(x) for x in d.counts)))
        return out
    return d, finish


def _grid(cfg) -> Grid:
    return Grid(nx=cfg.nx, ny=cfg.ny, dx_nm=cfg.dx_nm, dy_nm=cfg.dy_nm, dt_fs=cfg.dt_fs,
                rad_every=cfg.rad_every, seed=cfg.seed, cfl=cfg.cfl)


def _species(cfg, cap_e=0, cap_i=0) -> Species:
    return Species(n_ref_cm3=cfg.n_ref_cm3, w_ion=cfg.w_ion, m_ion_me=cfg.m_ion_me,
                   E_bulk_eV=cfg.E_bulk_eV, ipd_model=cfg.ipd_model, coulomb_log=cfg.coulomb_log,
                   flags=cfg.flags, cap_e=cap_e, cap_i=cap_i)


SLOT_FREE, SLOT_ACTIVE, SLOT_RETIRED, SLOT_FAILED = 0, 1, 2, 3


class Batch:
    """Many independent 1D slabs stepped together (one launch of each kernel
    per step), admitted and retired between steps."""

    def __init__(self, tables: dict, max_slabs: int, slot_cells: int, cap_e: int, cap_i: int, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise PicError("no CUDA device")
        self.L = lib()
        self.max_slabs, self.slot_cells = max_slabs, slot_cells
        check_capacity(cap_e, cap_i)
        self._t, self._keep = _tables(tables)
        nbytes = self.L.pic_batch_required_bytes(max_slabs, slot_cells, cap_e, cap_i)
        if nbytes == 0:
            raise PicError("pic_batch_required_bytes: invalid sizes")
        self.arena = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        s = stream if stream is not None else torch.cuda.current_stream()
        self.h = C.c_void_p()
        st = self.L.pic_batch_init(C.byref(self.h), max_slabs, slot_cells, cap_e, cap_i, C.byref(self._t),
                                   self.arena.data_ptr(), nbytes, s.cuda_stream)
        if st != 0:
            raise PicError(f"pic_batch_init: {STATUS.get(st, st)}")
        self.cfgs = {}

    _check = Slab._check
    close = Slab.close
    __del__ = Slab.__del__
    step = Slab.step
    sync = Slab.sync
    timing = Slab.timing
    launches = Slab.launches
    use_graphs = Slab.use_graphs
    autotune = Slab.autotune
    autotune = Slab.autotune

    def admit(self, cfg, st, pulse=None) -> int:
        g, sp = _grid(cfg), _species(cfg)
        pl = C.byref(pulse_struct(pulse)) if pulse is not None else None
        slot = C.c_int(-1)
        _ek, e = _electron_args(st)
        _ik, i = _ion_args(st)
        self._check(self.L.pic_batch_admit(self.h, C.byref(g), C.byref(sp), pl, *e, *i, C.byref(slot)),
                    "pic_batch_admit")
        self.cfgs[slot.value] = cfg
        return slot.value

    def retire(self, slot: int):
        self._check(self.L.pic_batch_retire(self.h, slot), "pic_batch_retire")
        self.cfgs.pop(slot, None)

    def set_budget(self, slot: int, max_e: int):
        """Electron budget of a slot (pic_batch_set_budget): beyond it the
        slab alone fails (state FAILED after the step), not the batch."""
        self._check(self.L.pic_batch_set_budget(self.h, slot, int(max_e)), "pic_batch_set_budget")

    def failed(self) -> list:
        """Slots that went beyond their electron budget (state FAILED)."""
        return [k for k in list(self.cfgs) if self.slot(k, step=False)[0] == SLOT_FAILED]

    def slot(self, slot: int, step: bool = True):
        state, n = C.c_int(), C.c_uint32()
        self._check(self.L.pic_batch_slot(self.h, slot, C.byref(state), C.byref(n) if step else None),
                    "pic_batch_slot")
        return state.value, n.value

    def counts(self, slot: int):
        ne, ni = C.c_int64(), C.c_int64()
        self._check(self.L.pic_batch_counts(self.h, slot, C.byref(ne), C.byref(ni)), "pic_batch_counts")
        return ne.value, ni.value

    def electrons(self, slot: int):
        n, _ = self.counts(slot)
        d, args = _electron_out(n)
        self._check(self.L.pic_batch_get_electrons(self.h, slot, *args), "pic_batch_get_electrons")
        return d

    def ions(self, slot: int):
        _, n = self.counts(slot)
        d, args = _ion_out(n)
        self._check(self.L.pic_batch_get_ions(self.h, slot, *args), "pic_batch_get_ions")
        return d

    def diagnostics(self, slot: int, n_E=64, E_max=1e4):
        d, finish = _diag_out(n_E, E_max)
        self._check(self.L.pic_batch_diagnostics(self.h, slot, C.byref(d)), "pic_batch_diagnostics")
        return finish()


def philox_check(ctr: np.ndarray, key) -> np.ndarray:
    """Device Philox4x32-10 outputs for counters ctr [n,4] and key (k0, k1)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros_like(c)
    st = lib().pic_philox_check(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(o, C.c_uint32), c.shape[0])
    if st != 0:
        raise PicError(f"pic_philox_check: {STATUS.get(st, st)}")
    return o


def dd_sum_check(x: np.ndarray, fp64: bool = False) -> float:
    """Sum of FP32 terms in the device's double-float cell-sum arithmetic."""
    v = np.ascontiguousarray(x, dtype=np.float32)
    out = np.zeros(1)
    st = lib(fp64).pic_dd_sum_check(_p(v, C.c_float), v.size, _p(out))
    if st != 0:
        raise PicError(f"pic_dd_sum_check: {STATUS.get(st, st)}")
    return float(out[0])


def order_check(key: np.ndarray, ids: np.ndarray, rmax: int = 512) -> np.ndarray:
    """Device in-cell ordering of (key, id) entries by the sort of the cell
    kernel instance rmax (128, 512, 1024): positions -> entry index."""
    k = np.ascontiguousarray(key, dtype=np.uint64)
    i = np.ascontiguousarray(ids, dtype=np.uint64)
    o = np.zeros(k.size, dtype=np.uint16)
    st = lib().pic_order_check(_p(k, C.c_uint64), _p(i, C.c_uint64), k.size, rmax, _p(o, C.c_uint16))
    if st != 0:
        raise PicError(f"pic_order_check: {STATUS.get(st, st)}")
    return o.astype(np.int64)
