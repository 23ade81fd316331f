"""The C-ABI library loads and exports every symbol include/mgrit.h declares,
and its host-side argument checks work without a GPU (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(mgrit_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2104_09404_gb300 import build as B, mgrit as M
    if not os.path.exists(M.LIB_PATH):
        B.build()
    return M.load()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("mgrit_create", "mgrit_set_params", "mgrit_solve", "mgrit_serial_step",
                     "mgrit_residual", "mgrit_last_error", "mgrit_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_2104_09404_gb300 import mgrit as M
    assert set(declared_symbols()) <= set(M._SIGS)


def test_default_params(lib):
    from paper_2104_09404_gb300 import mgrit as M
    p = M.mgrit_params()
    lib.mgrit_default_params(ctypes.byref(p))
    assert (p.T, p.L, p.relax, p.cycle, p.guess, p.numflux) == (1.0, 1.0, 1, 0, 0, 0)
    assert p.tol == 1e-10 and p.max_iter == 64 and p.precision == 64 and p.coarse == 0
    assert p.chunk_clusters == 1 and p.seq_stepper == 0


@pytest.mark.parametrize("args,frag", [
    ((128, 256, 1, 2, 0, 0), "m must"),
    ((128, 256, 4, 1, 0, 0), "levels"),
    ((128, 250, 4, 2, 0, 0), "divisible"),
    ((128, 16, 4, 4, 0, 0), "divisible"),
    ((4, 256, 4, 2, 0, 0), "nx too small"),
    ((2, 256, 4, 2, 1, 0), "nx too small"),
    ((128, 256, 4, 2, 7, 0), "scheme"),
    ((128, 256, 4, 2, 0, 9), "flux"),
    ((1 << 15, 256, 4, 2, 0, 0), "slab limit"),
])
def test_create_rejects_bad_arguments(lib, args, frag):
    from paper_2104_09404_gb300 import mgrit as M
    h = ctypes.c_void_p()
    st = lib.mgrit_create(ctypes.byref(h), *args)
    assert st == M.EINVAL
    assert not h.value
    assert frag in lib.mgrit_last_error(None).decode()


def test_create_set_params_destroy_without_gpu(lib):
    from paper_2104_09404_gb300 import mgrit as M
    h = ctypes.c_void_p()
    assert lib.mgrit_create(ctypes.byref(h), 100, 64, 4, 3, 0, 0) == M.OK
    p = M.mgrit_params()
    lib.mgrit_default_params(ctypes.byref(p))
    p.T = 0.5
    assert lib.mgrit_set_params(h, ctypes.byref(p)) == M.OK
    for field, bad in (("relax", 3), ("cycle", 2), ("guess", 2), ("numflux", 5), ("coarse", 3),
                       ("coarse", 1),
                       ("tol", -1.0), ("max_iter", 1000), ("precision", 16), ("T", 0.0),
                       ("chunk_clusters", 3), ("seq_stepper", 4), ("seq_stepper", -1)):
        q = M.mgrit_params.from_buffer_copy(p)
        setattr(q, field, bad)
        assert lib.mgrit_set_params(h, ctypes.byref(q)) == M.EINVAL, field
    # 100 cells: FP64 WENO5 slabs take at least 4 cells per thread (interface quads)
    assert lib.mgrit_query(h, 0) == 4 and lib.mgrit_query(h, 1) == 32
    assert lib.mgrit_query(h, 2) == 0 and lib.mgrit_query(h, 9) == -1    # nothing allocated yet
    assert lib.mgrit_query(h, 3) == 0                                     # grid stepper unknown yet
    # chunk cluster sizes of levels 0 and 1 (3 levels): unknown before allocation
    assert lib.mgrit_query(h, 100) == 0 and lib.mgrit_query(h, 101) == 0
    assert lib.mgrit_query(h, 102) == -1 and lib.mgrit_query(h, 99) == -1
    # 3 levels, m = 4: (2*4 + 1) * 16 + (2*4 + 1 + 3) * 4 + 4 steps per cycle at FCF
    assert lib.mgrit_cycle_cell_updates(h) == 100 * ((2 * 4 + 1) * 16 + (2 * 4 + 1 + 3) * 4 + 4)
    # F-cycle: level 1 is visited twice (relaxation, coarsest solve, interpolation each time)
    q = M.mgrit_params.from_buffer_copy(p)
    q.cycle = M.CYCLE_F
    assert lib.mgrit_set_params(h, ctypes.byref(q)) == M.OK
    assert lib.mgrit_cycle_cell_updates(h) == 100 * ((2 * 4 + 1) * 16 + 2 * ((2 * 4 + 1 + 3) * 4 + 4))
    lib.mgrit_destroy(h)
    lib.mgrit_destroy(None)


def test_null_arguments_are_rejected(lib):
    from paper_2104_09404_gb300 import mgrit as M
    assert lib.mgrit_create(None, 100, 64, 4, 3, 0, 0) == M.EINVAL
    assert lib.mgrit_solve(None, None, None, None, None, None) == M.EINVAL
    assert lib.mgrit_serial_step(None, None, None, 1, None) == M.EINVAL
    h = ctypes.c_void_p()
    assert lib.mgrit_create(ctypes.byref(h), 100, 64, 4, 3, 0, 0) == M.OK
    assert lib.mgrit_solve(h, None, None, None, None, None) == M.EINVAL
    assert lib.mgrit_copy_cpoints(h, None, None) == M.EINVAL
    lib.mgrit_destroy(h)


def test_adjoint_shape_and_host_checks_without_gpu(lib):
    from paper_2104_09404_gb300 import mgrit as M
    h = ctypes.c_void_p()
    assert lib.mgrit_create(ctypes.byref(h), 2048, 64, 4, 2, 0, 0) == M.OK
    assert lib.mgrit_adjoint_query(h, 0) == 4 and lib.mgrit_adjoint_query(h, 1) == 512
    assert lib.mgrit_adjoint_query(h, 7) == -1
    lib.mgrit_destroy(h)
    # nx above the one-CTA adjoint slab (4096): no one-CTA shape; the adjoint
    # then runs on clusters, chosen at the first adjoint call
    assert lib.mgrit_create(ctypes.byref(h), 8192, 64, 4, 2, 0, 0) == M.OK
    assert lib.mgrit_adjoint_query(h, 0) == 0 and lib.mgrit_adjoint_query(h, 1) == 0
    assert lib.mgrit_adjoint_query(h, 2) == 0 and lib.mgrit_adjoint_query(h, 100) == 0
    assert lib.mgrit_adjoint_query(h, 101) == -1     # 2 levels: only level 0 has chunks
    lib.mgrit_destroy(h)
    one = ctypes.c_void_p(16)   # never dereferenced: the flux check comes first
    # the state-reconstruction flux has no adjoint
    assert lib.mgrit_create(ctypes.byref(h), 256, 64, 4, 2, 0, 0) == M.OK
    p = M.mgrit_params()
    lib.mgrit_default_params(ctypes.byref(p))
    p.numflux = 1
    assert lib.mgrit_set_params(h, ctypes.byref(p)) == M.OK
    assert lib.mgrit_adjoint_query(h, 0) == 0
    st = lib.mgrit_step_vjp(h, one, one, one, None)
    assert st == M.EINVAL and "split" in lib.mgrit_last_error(h).decode()
    lib.mgrit_destroy(h)


def test_lf_scheme_host_checks_without_gpu(lib):
    from paper_2104_09404_gb300 import mgrit as M
    h = ctypes.c_void_p()
    assert lib.mgrit_create(ctypes.byref(h), 128, 1024, 2, 5, M.LF_FE, M.BURGERS) == M.OK
    p = M.mgrit_params()
    lib.mgrit_default_params(ctypes.byref(p))
    for coarse in (M.COARSE_REDISC, M.COARSE_PSI0, M.COARSE_PSI1):
        p.coarse = coarse
        assert lib.mgrit_set_params(h, ctypes.byref(p)) == M.OK
    p.precision = 32
    assert lib.mgrit_set_params(h, ctypes.byref(p)) == M.EINVAL
    assert "FP64 only" in lib.mgrit_last_error(h).decode()
    assert lib.mgrit_adjoint_query(h, 0) == 0
    lib.mgrit_destroy(h)
    assert lib.mgrit_create(ctypes.byref(h), 2, 64, 2, 2, M.LF_FE, M.BURGERS) == M.EINVAL


def test_slice_width_limits_without_gpu(lib):
    # one CTA holds 8192 FP64 or 16384 FP32 cells; wider FP64 slices run
    # every chunk on a thread-block cluster (up to 16 CTAs x 1024 cells),
    # except under the classical LF scheme, which has one-CTA kernels only
    from paper_2104_09404_gb300 import mgrit as M
    h = ctypes.c_void_p()
    p = M.mgrit_params()
    for nx in (8193, 16384):
        assert lib.mgrit_create(ctypes.byref(h), nx, 64, 2, 2, M.WENO5_SSPRK3, M.BURGERS) == M.OK
        lib.mgrit_default_params(ctypes.byref(p))
        assert lib.mgrit_set_params(h, ctypes.byref(p)) == M.OK       # FP64 sweeps
        p.precision = 32
        assert lib.mgrit_set_params(h, ctypes.byref(p)) == M.OK
        lib.mgrit_destroy(h)
    assert lib.mgrit_create(ctypes.byref(h), 16385, 64, 2, 2, M.WENO5_SSPRK3, M.BURGERS) == M.EINVAL
    assert lib.mgrit_create(ctypes.byref(h), 8193, 64, 2, 2, M.LF_FE, M.BURGERS) == M.EINVAL
    assert lib.mgrit_create(ctypes.byref(h), 8192, 64, 2, 2, M.LF_FE, M.BURGERS) == M.OK
    lib.mgrit_destroy(h)


def _header_struct_fields(name):
    # (type, field) pairs of `typedef struct { ... } name;` in include/mgrit.h,
    # in declaration order (comments removed; "int a, b;" gives two fields)
    src = open(os.path.join(ROOT, "include", "mgrit.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", src).group(1)
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        ctype, names = decl.split(None, 1)
        for n in names.split(","):
            n = n.strip()
            m = re.match(r"(\w+)\s*\[(\d+)\]", n)
            out.append((ctype, m.group(1), int(m.group(2))) if m else (ctype, n, 1))
    return out


@pytest.mark.parametrize("name", ["mgrit_params", "mgrit_stats", "mgrit_instance"])
def test_binding_structs_match_the_header(name):
    # the ctypes mirrors declare the header's fields in the header's order
    # with the same C types, so the layouts (and sizes) agree
    from paper_2104_09404_gb300 import mgrit as M
    ctypes_of = {"double": ctypes.c_double, "int": ctypes.c_int}
    cls = getattr(M, name)
    want = _header_struct_fields(name)
    got = list(cls._fields_)
    assert [f for f, _ in got] == [n for _, n, _ in want]
    for (fname, ftype), (ctype, _, count) in zip(got, want):
        base = ctypes_of[ctype]
        assert ftype == (base * count if count > 1 else base), fname
