"""The C ABI's host-side contract, without a GPU: the arena sizing of
pic_required_bytes / pic_batch_required_bytes (bytes per particle slot as
the HBM layout states them, the large 2D slab's arena within one GB300),
the refusal of invalid grids, species and sizes, and the PIC_ERR_ARG answer
of every call to a NULL context or out-of-range size, all of which the
library checks before it touches the device (no CUDA call is made here),
and the binding's ctypes signatures against the header's prototypes."""
import ctypes as C

import numpy as np
import pytest

import pic_inputs as P
import paper_1704_01202_gb300 as pkg
from paper_1704_01202_gb300 import Grid, Species, Tables, _grid, _species

PIC_OK, PIC_ERR_ARG = 0, 1
GIB = 1 << 30


@pytest.fixture(scope="module", params=[False, True], ids=["fp32", "fp64"])
def build(request):
    pkg.build()
    L = pkg.lib(request.param)
    return L, (8 if request.param else 4)


def _req(L, cfg, ce, ci):
    g, s = _grid(cfg), _species(cfg)
    return L.pic_required_bytes(C.byref(g), C.byref(s), ce, ci)


def test_arena_bytes_per_particle_slot(build):
    """Each electron or ion slot costs two records of four reals, double
    buffered for the scatter, plus the 4 B next-cell key: 68 B in the FP32
    build, 132 B in the FP64 build."""
    L, rb = build
    cfg = P.cfg_small_1d()
    base = _req(L, cfg, 64 * 1024, 64 * 1024)
    per_slot = 2 * 2 * 4 * rb + 4
    assert _req(L, cfg, 64 * 1024 + 6400, 64 * 1024) - base == 6400 * per_slot
    assert _req(L, cfg, 64 * 1024, 64 * 1024 + 6400) - base == 6400 * per_slot


def test_large_slab_arena_fits_one_gb300(build):
    """8192 x 1024 cells with 80 e + 20 i per cell and electron room for a
    mean charge of 9.5: ~129 GB in the FP32 build, within the GPU's 284,208
    MiB with room for the rest of the process."""
    L, rb = build
    cfg = P.cfg_large_2d()
    n_i = cfg.ncell * cfg.ppc_i
    ce, ci = int(9.5 * n_i) + 1024, n_i + 1024
    b = _req(L, cfg, ce, ci)
    if rb == 4:
        assert 120e9 < b < 140e9, b / 1e9
        assert b < 0.5 * 284208 * (1 << 20)
    else:
        assert b > 1.9 * 120e9         # the FP64 check build is not sized for this slab


def test_required_bytes_refuses_invalid_grids(build):
    L, _ = build
    cfg = P.cfg_small_1d()
    s = _species(cfg)
    assert L.pic_required_bytes(None, C.byref(s), 1024, 256) == 0
    assert L.pic_required_bytes(C.byref(_grid(cfg)), None, 1024, 256) == 0
    for field, value in (("nx", 1), ("nx", 8193), ("ny", 0), ("dx_nm", 0.0), ("dy_nm", -1.0),
                         ("dt_fs", 0.0), ("cfl", 0.0)):
        g = _grid(cfg)
        setattr(g, field, value)
        assert L.pic_required_bytes(C.byref(g), C.byref(s), 1024, 256) == 0, field
    g = _grid(cfg)
    g.nx, g.ny = 8191, (1 << 27) // 8192 + 1          # more than 2^27 grid points
    assert L.pic_required_bytes(C.byref(g), C.byref(s), 1024, 256) == 0
    g.ny = (1 << 27) // 8192
    assert L.pic_required_bytes(C.byref(g), C.byref(s), 1024, 256) > 0
    assert L.pic_batch_required_bytes((1 << 27) // 4097 + 1, 4096, 1024, 256) == 0
    assert L.pic_batch_required_bytes((1 << 27) // 4097, 4096, 1024, 256) > 0


def test_batch_required_bytes(build):
    L, _ = build
    for args in ((0, 64, 1000, 250), (4, 1, 1000, 250), (4, 8193, 1000, 250), (4, 64, 0, 250), (4, 64, 1000, 0)):
        assert L.pic_batch_required_bytes(*args) == 0, args
    one = L.pic_batch_required_bytes(4, 64, 64 * 100, 64 * 25)
    assert one > 0
    assert L.pic_batch_required_bytes(4, 8192, 64 * 100, 64 * 25) > one
    assert L.pic_batch_required_bytes(4, 64, 64 * 200, 64 * 25) > one


def test_init_refuses_before_touching_the_device(build):
    L, _ = build
    cfg = P.cfg_small_1d()
    tabs = Tables()
    ctx = C.c_void_p(123)
    g_bad = _grid(cfg)
    g_bad.nx = 1
    s = _species(cfg, 4096, 1024)
    assert L.pic_init(C.byref(ctx), C.byref(g_bad), C.byref(s), C.byref(tabs), None, 0, None) == PIC_ERR_ARG
    assert ctx.value is None
    s0 = _species(cfg, 0, 1024)
    assert L.pic_init(C.byref(ctx), C.byref(_grid(cfg)), C.byref(s0), C.byref(tabs), None, 0, None) == PIC_ERR_ARG
    assert L.pic_init(C.byref(ctx), C.byref(_grid(cfg)), C.byref(s), None, None, 0, None) == PIC_ERR_ARG
    bad_s = _species(cfg, 4096, 1024)
    bad_s.w_ion = 0.0
    assert L.pic_init(C.byref(ctx), C.byref(_grid(cfg)), C.byref(bad_s), C.byref(tabs), None, 0,
                      None) == PIC_ERR_ARG
    assert L.pic_batch_init(C.byref(ctx), 4, 1, 1000, 250, C.byref(tabs), None, 0, None) == PIC_ERR_ARG
    assert L.pic_batch_init(C.byref(ctx), 4, 64, 1000, 250, None, None, 0, None) == PIC_ERR_ARG


def test_null_context_calls(build):
    L, _ = build
    n = C.c_int64()
    for name, args in (("pic_step", (None, 1)), ("pic_sync", (None,)), ("pic_diagnostics", (None, None)),
                       ("pic_counts", (None, C.byref(n), C.byref(n))), ("pic_free", (None,)),
                       ("pic_source", (None, None)), ("pic_seed", (None, None)),
                       ("pic_checkpoint", (None, None, 0)), ("pic_restore", (None, None, 0)),
                       ("pic_get_photons", (None, None)), ("pic_rt_get", (None, None, None, None)),
                       ("pic_batch_retire", (None, 0)), ("pic_batch_set_budget", (None, 0, 10)),
                       ("pic_batch_slot", (None, 0, None, None)), ("pic_use_graphs", (None, 1)),
                       ("pic_autotune", (None, 1, None, None)), ("pic_timing", (None, 1, None, None))):
        assert getattr(L, name)(*args) == PIC_ERR_ARG, name
    assert L.pic_checkpoint_bytes(None) == 0
    assert L.pic_launch_count(None) == 0
    assert L.pic_last_error(None) == b"no context"


def test_size_returning_calls_keep_their_width(build):
    """The binding declares every size_t / int64 result as such, so a
    checkpoint image or an arena past 2 GiB is not truncated."""
    L, _ = build
    for name in ("pic_required_bytes", "pic_batch_required_bytes", "pic_checkpoint_bytes"):
        assert getattr(L, name).restype is C.c_size_t, name
    assert L.pic_launch_count.restype is C.c_int64
    cfg = P.cfg_large_2d()
    assert _req(L, cfg, 1 << 30, 1 << 28) > 4 * GIB


def test_check_entries_refuse_bad_sizes(build):
    L, _ = build
    u32 = np.zeros(4 * 8, dtype=np.uint32)
    p32 = u32.ctypes.data_as(C.POINTER(C.c_uint32))
    assert L.pic_philox_check(p32, p32, p32, 0) == PIC_ERR_ARG
    assert L.pic_philox_check_static(p32, p32, p32, 0) == PIC_ERR_ARG
    assert L.pic_philox_check_static(p32, p32, p32, 4097) == PIC_ERR_ARG
    k = np.zeros(8, dtype=np.uint64)
    pk = k.ctypes.data_as(C.POINTER(C.c_uint64))
    o = np.zeros(8, dtype=np.uint16)
    po = o.ctypes.data_as(C.POINTER(C.c_uint16))
    for n, rmax in ((8, 256), (129, 128), (4097, 1024), (0, 512)):
        assert L.pic_order_check(pk, pk, n, rmax, po) == PIC_ERR_ARG, (n, rmax)
    x = np.zeros(4, dtype=np.float32)
    d = C.c_double()
    px = x.ctypes.data_as(C.POINTER(C.c_float))
    assert L.pic_dd_sum_check(px, 0, C.byref(d)) == PIC_ERR_ARG
    assert L.pic_dd_sum_check(px, (1 << 24) + 1, C.byref(d)) == PIC_ERR_ARG


def _prototypes():
    """(result type, [parameter types]) of every function include/pic.h
    declares, comments removed and whitespace normalized."""
    import os
    import re
    src = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "pic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"([A-Za-z_][\w \*]*?)\b(pic_\w+)\s*\(([^;{]*?)\)\s*;", src):
        ret, name, params = " ".join(m.group(1).split()), m.group(2), " ".join(m.group(3).split())
        types = []
        for p in ([] if params in ("", "void") else params.split(",")):
            p = p.strip()
            arr = p.endswith("]")
            p = re.sub(r"\[\d*\]$", "", p)
            t = re.sub(r"\b\w+$", "", p).replace(" ", "").replace("const", "")
            types.append(t + ("*" if arr else ""))
        out[name] = (ret.replace("const ", "").replace(" ", ""), types)
    return out


_CTYPE = {"int": C.c_int, "int64_t": C.c_int64, "size_t": C.c_size_t, "void*": C.c_void_p,
          "pic_ctx*": C.c_void_p, "pic_ctx**": C.POINTER(C.c_void_p), "double*": C.POINTER(C.c_double),
          "float*": C.POINTER(C.c_float), "uint64_t*": C.POINTER(C.c_uint64),
          "uint32_t*": C.POINTER(C.c_uint32), "int32_t*": C.POINTER(C.c_int32),
          "uint16_t*": C.POINTER(C.c_uint16), "int*": C.POINTER(C.c_int), "int64_t*": C.POINTER(C.c_int64),
          "pic_grid*": C.POINTER(Grid), "pic_species*": C.POINTER(Species), "pic_tables*": C.POINTER(Tables),
          "pic_pulse*": C.POINTER(pkg.Pulse), "pic_diag*": C.POINTER(pkg.Diag),
          "pic_seed_spec*": C.POINTER(pkg.SeedSpec), "pic_rt_config*": C.POINTER(pkg.RTConfig)}
_RTYPE = {"pic_status": C.c_int, "int": C.c_int, "size_t": C.c_size_t, "int64_t": C.c_int64, "char*": C.c_char_p}


def test_binding_signatures_match_the_header(build):
    """Every function's ctypes argument and result types in the binding
    are the ones its C prototype gives (a narrower integer or a wrong
    pointer type would corrupt values silently)."""
    L, _ = build
    protos = _prototypes()
    assert sorted(protos) == sorted(pkg.ABI_FUNCTIONS)
    for name, (ret, params) in protos.items():
        f = getattr(L, name)
        assert f.restype is _RTYPE[ret], (name, ret, f.restype)
        if not params:
            continue
        assert f.argtypes is not None, name
        want = [_CTYPE[t] for t in params]
        assert list(f.argtypes) == want, (name, params, f.argtypes)


def test_capacities_stay_within_32_bit_particle_indices(build):
    """cap_e + 3 cap_i must stay below 2^31 (a step appends at most three
    electrons per ion after the held ones): the library refuses beyond, at
    pic_required_bytes, pic_init and pic_batch_required_bytes, and the
    binding refuses before a value can wrap in a 32-bit ctypes field."""
    L, _ = build
    cfg = P.cfg_small_1d()
    top = (1 << 31) - 1
    ci = 1 << 20
    assert _req(L, cfg, top - 3 * ci, ci) > 0
    assert _req(L, cfg, top - 3 * ci + 1, ci) == 0
    assert L.pic_batch_required_bytes(2, 64, top - 3 * ci, ci) > 0
    assert L.pic_batch_required_bytes(2, 64, top - 3 * ci + 1, ci) == 0
    ctx = C.c_void_p()
    s = _species(cfg, top - 3 * ci + 1, ci)
    assert L.pic_init(C.byref(ctx), C.byref(_grid(cfg)), C.byref(s), C.byref(Tables()), None, 0,
                      None) == PIC_ERR_ARG
    pkg.check_capacity(top - 3 * ci, ci)
    for ce, c_i in ((top - 3 * ci + 1, ci), (4_500_000_000, 1000), (0, 10), (10, 0), (-5, 10)):
        with pytest.raises(pkg.PicError, match="capacity"):
            pkg.check_capacity(ce, c_i)


def test_bench_capacity_of_the_large_slab():
    import importlib.util
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_cap", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    cfg = P.cfg_large_2d()
    n_e, n_i = cfg.ncell * cfg.ppc_e, cfg.ncell * cfg.ppc_i
    ce, ci = bench.capacity(cfg, n_e, n_i)
    assert ce == int(9.5 * n_i) + 1024 and ci == n_i + 1024     # room for a mean charge of 9.5
    pkg.check_capacity(ce, ci)


def test_non_finite_inputs_are_refused(build):
    """Cell sizes, steps and Courant numbers must be finite, and so must the
    species' weights, masses, densities and Coulomb logarithm: pic_init
    refuses before anything reaches the device."""
    L, _ = build
    cfg = P.cfg_small_1d()
    tabs = Tables()
    ctx = C.c_void_p()
    for field in ("dx_nm", "dy_nm", "dt_fs", "cfl"):
        for v in (float("inf"), float("nan")):
            g = _grid(cfg)
            setattr(g, field, v)
            assert _req_g(L, g, cfg) == 0, (field, v)
            assert L.pic_init(C.byref(ctx), C.byref(g), C.byref(_species(cfg, 4096, 1024)), C.byref(tabs),
                              None, 0, None) == PIC_ERR_ARG, (field, v)
    for field in ("w_ion", "m_ion_me", "n_ref_cm3", "coulomb_log", "E_bulk_eV"):
        s = _species(cfg, 4096, 1024)
        setattr(s, field, float("nan"))
        assert L.pic_init(C.byref(ctx), C.byref(_grid(cfg)), C.byref(s), C.byref(tabs), None, 0,
                          None) == PIC_ERR_ARG, field


def _req_g(L, g, cfg):
    s = _species(cfg)
    return L.pic_required_bytes(C.byref(g), C.byref(s), 1024, 256)


def test_particle_arrays_of_unequal_length_are_refused():
    """The binding passes one count for all of a species' arrays: arrays of
    another length are refused before the library could read past them."""
    cfg = P.cfg_small_1d(nx=4, ppc_e=4, ppc_i=1)
    st = P.init_particles(cfg)
    pkg._electron_args(st)
    pkg._ion_args(st)
    for field, cut in (("eY", slice(0, -1)), ("ew", slice(0, -1)), ("eid", slice(0, -1)), ("eu", slice(0, -1))):
        bad = P.init_particles(cfg)
        setattr(bad, field, getattr(bad, field)[cut])
        with pytest.raises(pkg.PicError, match="lengths"):
            pkg._electron_args(bad)
    bad = P.init_particles(cfg)
    bad.eu = bad.eu[:, :2]
    with pytest.raises(pkg.PicError, match="lengths"):
        pkg._electron_args(bad)
    for field in ("iY", "izf", "iZ", "inK", "iid", "iu"):
        bad = P.init_particles(cfg)
        setattr(bad, field, getattr(bad, field)[:-1])
        with pytest.raises(pkg.PicError, match="lengths"):
            pkg._ion_args(bad)


def test_setters_refuse_arrays_of_another_size():
    """Photon numbers, fields and the rad field are read by count: a wrong
    size is refused in the binding, before the library is called (the slab
    here has no context at all)."""
    cfg = P.cfg_small_1d(nx=8)
    s = object.__new__(pkg.Slab)
    s.cfg, s.n_bins, s.L, s.h = cfg, 2, None, None
    s.nord, s.nry, s.nrx = 3, 1, 4
    with pytest.raises(pkg.PicError, match="photon numbers"):
        s.set_photons(np.zeros((cfg.ny, cfg.nx, 3)))
    f = P.random_fields(cfg, 1)
    f["ez"] = f["ez"][:, :-1]
    with pytest.raises((pkg.PicError, ValueError)):
        s.set_fields(f)
    f = {k: np.zeros((cfg.ny, cfg.nx)) for k in ("ex", "ey", "ez", "bx", "by", "bz")}
    with pytest.raises(pkg.PicError, match="fields"):
        s.set_fields(f)
    with pytest.raises(pkg.PicError, match="rad field F"):
        s.set_rt_field(np.zeros((3, 2, 1, 5)))
    with pytest.raises(pkg.PicError, match="rad field Gy"):
        s.set_rt_field(np.zeros((3, 2, 1, 4)), np.zeros((3, 2, 1, 4)), np.zeros(3))
