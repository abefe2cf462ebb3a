"""The C ABI library: it builds for sm_103a, loads without a GPU, exports every function
that include/lbm2p.h declares, and rejects bad parameters before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1808_07554_gb300 import build
    build.build()
    import paper_1808_07554_gb300 as pkg
    return pkg.load_library()


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(lbm2p_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_abi_version_and_defaults(lib):
    import paper_1808_07554_gb300 as pkg
    assert pkg.lbm2p_abi_version() == 7
    p = pkg.lbm2p_default_params()
    assert (p.phi, p.beta, p.mu_w, p.mu_n, p.D_s, p.tau_p, p.tol) == (0.2, 0.4, 1.0, 2.0, 0.01, 1.0, 1e-8)
    assert p.check_every == 8 and list(p.bc) == [1, 1, 1, 1] and p.fuse_sweeps == 0
    assert p.sweep_kernel == pkg.SWEEP_AUTO and p.sat_lattice == 9 and p.D_c == 0.0
    assert p.warm_start == 0


def _inputs(pkg, n, K=None, S0=None):
    inp = pkg.lbm2p_inputs()
    K = np.ones(n) if K is None else K
    S0 = np.full(n, 0.2) if S0 is None else S0
    inp.K = K.ctypes.data_as(C.POINTER(C.c_double))
    inp.S0 = S0.ctypes.data_as(C.POINTER(C.c_double))
    return inp, (K, S0)


@pytest.mark.parametrize("field,value,status", [
    ("nx", 0, 1), ("dx", -1.0, 1), ("phi", 0.0, 1), ("D_s", 0.0, 1), ("tau_p", 0.5, 1),
    ("check_every", 0, 1), ("max_sub_iters", 0, 1), ("storage", 2, 1), ("mobility", 9, 1),
    ("tol", -1.0, 1), ("fuse_sweeps", 3, 1), ("sweep_kernel", 4, 1), ("sweep_kernel", -1, 1), ("sat_lattice", 7, 1),
    ("D_c", -1.0, 1), ("warm_start", 2, 1)])
def test_bad_parameters_are_rejected_without_a_device(lib, field, value, status):
    import paper_1808_07554_gb300 as pkg
    p = pkg.lbm2p_default_params()
    p.nx = p.ny = 8
    setattr(p, field, value)
    inp, keep = _inputs(pkg, 64)
    h = C.c_void_p()
    st = lib.lbm2p_create(C.byref(h), C.byref(p), C.byref(inp), None)
    assert st == status and not h.value
    assert len(pkg.lbm2p_last_error(None)) > 0


def test_bad_walls_wells_and_fields_are_rejected(lib):
    import paper_1808_07554_gb300 as pkg
    p = pkg.lbm2p_default_params()
    p.nx = p.ny = 8
    p.bc[0] = pkg.PERIODIC                      # unpaired periodic side
    inp, keep = _inputs(pkg, 64)
    h = C.c_void_p()
    assert lib.lbm2p_create(C.byref(h), C.byref(p), C.byref(inp), None) == pkg.EINVAL
    p.bc[0] = pkg.NOFLUX
    K = np.ones(64)
    K[5] = -1.0                                 # non-positive permeability
    inp, keep = _inputs(pkg, 64, K=K)
    assert lib.lbm2p_create(C.byref(h), C.byref(p), C.byref(inp), None) == pkg.EINVAL
    assert "K must be positive" in pkg.lbm2p_last_error(None)
    inp, keep = _inputs(pkg, 64)
    w = (pkg.lbm2p_well * 1)(pkg.lbm2p_well(8, 0, 1e-3, 0))    # outside the lattice
    inp.wells = C.cast(w, C.POINTER(pkg.lbm2p_well))
    inp.n_wells = 1
    assert lib.lbm2p_create(C.byref(h), C.byref(p), C.byref(inp), None) == pkg.EINVAL
    p.bc[0] = p.bc[1] = pkg.DIRICHLET
    p.nx = 2
    inp, keep = _inputs(pkg, 16)
    assert lib.lbm2p_create(C.byref(h), C.byref(p), C.byref(inp), None) == pkg.EINVAL
    assert not h.value


def test_null_handle_calls_fail_cleanly(lib):
    import paper_1808_07554_gb300 as pkg
    assert lib.lbm2p_step(None, 1, None, None) == pkg.EINVAL
    assert lib.lbm2p_fields(None, None, None, 0, 0) == pkg.EINVAL
    assert lib.lbm2p_state_count(None) == 0
    assert lib.lbm2p_fused_form_of(None) == pkg.FUSED_NONE
    assert lib.lbm2p_set_fused_shape(None, pkg.FUSED_STAGED_ROWS, 4, 6, 16) == pkg.EINVAL
    lib.lbm2p_destroy(None)


def test_binding_constants_match_the_header():
    import paper_1808_07554_gb300 as pkg
    text = open(os.path.join(ROOT, "include", "lbm2p.h")).read()
    m = re.search(r"#define\s+LBM2P_NOALLOC_MAX_TILES\s+(\d+)", text)
    assert m and int(m.group(1)) == pkg.NOALLOC_MAX_TILES
    assert "row tile of 1024" in text and pkg.NOALLOC_TILE_NODES == 1024
    m = re.search(r"#define\s+LBM2P_MAX_WELLS\s+(\d+)", text)
    assert m and int(m.group(1)) == pkg.MAX_WELLS
    m = re.search(r"#define\s+LBM2P_ROWS2_DENSE\s+(\d+)", text)
    assert m and int(m.group(1)) == pkg.ROWS2_DENSE


def _cuda_present():
    try:
        import torch
        return torch.cuda.is_available()
    except ImportError:
        return False


@pytest.mark.skipif(_cuda_present(), reason="host-only check: it passes addresses that are not "
                                            "device memory, so it never runs where a GPU is")
def test_noalloc_rejects_aliased_planes_before_any_cuda_call(lib):
    """The argument checks of the allocation-free sweep come before its first CUDA call, so
    on a machine without a GPU a rejected call returns EINVAL with its reason."""
    import paper_1808_07554_gb300 as pkg
    planes_in = [4096 * (i + 1) for i in range(8)]
    planes_out = [4096 * (i + 20) for i in range(8)]
    R, it, dP = 4096 * 40, 4096 * 41, 4096 * 42
    bad = list(planes_out)
    bad[3] = planes_in[5]                      # an output plane that is an input plane
    with pytest.raises(pkg.LBM2PError) as ei:
        pkg.lbm2p_pressure_sweep_noalloc(64, 64, 64, (1, 1, 1, 1), planes_in, bad, R, it, 0,
                                         None, dP)
    assert ei.value.status == pkg.EINVAL and "n_in[5]" in str(ei.value)
    bad = list(planes_out)
    bad[0] = bad[7]                            # two outputs on one plane
    with pytest.raises(pkg.LBM2PError) as ei:
        pkg.lbm2p_pressure_sweep_noalloc(64, 64, 64, (1, 1, 1, 1), planes_in, bad, R, it, 0,
                                         None, dP)
    assert ei.value.status == pkg.EINVAL
    with pytest.raises(pkg.LBM2PError) as ei:  # the increment plane on the reference pressure
        pkg.lbm2p_pressure_sweep_noalloc(64, 64, 64, (1, 1, 1, 1), planes_in, planes_out, R, it,
                                         0, None, R)
    assert ei.value.status == pkg.EINVAL and "dP" in str(ei.value)
