"""The C-ABI library loads and exports every symbol include/mujica_pm.h
declares; host-side validation and host coefficients (no GPU needed)."""
import ctypes
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

from oracle import cosmology as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_26823_gb300 import build, _lib
    build.build()
    return _lib.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "mujica_pm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pm_\w+|lbfgs_\w+|project_rank_match)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "pm_forward" in names and "pm_adjoint" in names and "lbfgs_step" in names
    assert "project_rank_match" in names
    for n in names:
        assert hasattr(lib, n), n
    from paper_2604_26823_gb300 import _lib
    assert set(names) == set(_lib.SIGNATURES), set(names) ^ set(_lib.SIGNATURES)


def test_config_struct_layout_matches_header(lib, tmp_path):
    """The binding's pm_config has the size and field offsets a C compiler
    gives the header's struct."""
    from paper_2604_26823_gb300 import _lib
    assert lib.pm_version().decode().startswith("mujica-pm")
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f for f, _ in _lib.pm_config._fields_]
    src = tmp_path / "layout.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"mujica_pm.h\"\nint main(void) {\n"
                   '  printf("size %zu\\n", sizeof(pm_config));\n'
                   + "".join(f'  printf("{f} %zu\\n", offsetof(pm_config, {f}));\n' for f in fields)
                   + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    assert int(out["size"]) == ctypes.sizeof(_lib.pm_config)
    for f in fields:
        assert int(out[f]) == getattr(_lib.pm_config, f).offset, f


def test_validation_errors_without_gpu(lib):
    from paper_2604_26823_gb300 import _lib, api
    cfg = api.Config(n=48, box=100.0).to_c()
    nb = ctypes.c_size_t()
    assert lib.pm_workspace_bytes(ctypes.byref(cfg), ctypes.byref(nb)) == 2   # UNSUPPORTED
    assert b"power of two" in lib.pm_last_error()
    cfg = api.Config(n=32, box=-1.0).to_c()
    assert lib.pm_workspace_bytes(ctypes.byref(cfg), ctypes.byref(nb)) == 1
    cfg = api.Config(n=32, box=128.0, likelihood="poisson", nbar_cell=0.0).to_c()
    assert lib.pm_workspace_bytes(ctypes.byref(cfg), ctypes.byref(nb)) == 1
    cfg = api.Config(n=32, box=128.0, bias="powerlaw_sigmoid", nbar_cell=0.0).to_c()
    assert lib.pm_workspace_bytes(ctypes.byref(cfg), ctypes.byref(nb)) == 1
    assert b"power-law bias" in lib.pm_last_error()
    cfg = api.Config(n=32, box=128.0, bias="linear", nbar_cell=0.0).to_c()   # Gaussian, linear: no nbar
    assert lib.pm_workspace_bytes(ctypes.byref(cfg), ctypes.byref(nb)) == 0
    cfg = api.Config(n=32, box=128.0).to_c()
    cfg.bias = 3
    assert lib.pm_workspace_bytes(ctypes.byref(cfg), ctypes.byref(nb)) == 1
    cfg = api.Config(n=32, box=128.0).to_c()
    assert lib.pm_workspace_bytes(ctypes.byref(cfg), ctypes.byref(nb)) == 0
    assert nb.value > 0
    # a plan with a too-small workspace is refused before any device call
    h = ctypes.c_void_p()
    lnk = np.linspace(-9, 4, 8)
    lnp = np.zeros(8)
    st = lib.pm_plan_create(ctypes.byref(cfg), lnk.ctypes.data_as(_lib._DP), lnp.ctypes.data_as(_lib._DP), 8,
                            ctypes.c_void_p(256), 1024, ctypes.byref(h))
    assert st == 5
    st = lib.lbfgs_workspace_bytes(100, 0, 0, ctypes.byref(nb))
    assert st == 1


def test_checkpoint_layout_is_smaller_at_large_step_counts(lib):
    from paper_2604_26823_gb300 import api
    nb0, nb2 = ctypes.c_size_t(), ctypes.c_size_t()
    c0 = api.Config(n=64, box=256.0, n_steps=10).to_c()
    c2 = api.Config(n=64, box=256.0, n_steps=10, checkpoint_every=2).to_c()
    assert lib.pm_workspace_bytes(ctypes.byref(c0), ctypes.byref(nb0)) == 0
    assert lib.pm_workspace_bytes(ctypes.byref(c2), ctypes.byref(nb2)) == 0
    assert nb2.value < nb0.value


def test_host_growth_matches_oracle(lib):
    from paper_2604_26823_gb300 import api
    a = np.array([0.1, 0.19, 0.55, 1.0])
    for om in (0.25, 1.0):
        got = api.pm_growth(om, a)
        ref = C.growth(a, om)
        for k in ("D1", "D2", "Gp1", "Gp2"):
            np.testing.assert_allclose(got[k], ref[k], rtol=1e-10)


def test_host_distance_table_matches_oracle(lib):
    from paper_2604_26823_gb300 import api
    for om in (0.25, 0.3):
        a, chi = api.pm_distance_table(om, 0.5, 257)
        ra, rchi = C.distance_table(om, 0.5, 257)
        np.testing.assert_allclose(a, ra, rtol=0, atol=1e-15)
        np.testing.assert_allclose(chi, rchi, rtol=1e-12, atol=1e-10)


def test_lightcone_validation_without_gpu(lib):
    from paper_2604_26823_gb300 import api
    nb = ctypes.c_size_t()
    ok = dict(n=32, box=128.0, n_steps=9, a_init=0.1, rsd_axis=3, observer=(64.0, 64.0, -260.0), lightcone=True)
    assert lib.pm_workspace_bytes(ctypes.byref(api.Config(**ok).to_c()), ctypes.byref(nb)) == 0
    with_lc = nb.value
    assert lib.pm_workspace_bytes(ctypes.byref(api.Config(**dict(ok, lightcone=False)).to_c()),
                                  ctypes.byref(nb)) == 0
    assert with_lc - nb.value >= 12 * 32 ** 3 * 4    # four snapshot arrays of 3 x n^3
    # no state at a = 0.8 / 0.9 on a 10-step grid from a = 0.1
    assert lib.pm_workspace_bytes(ctypes.byref(api.Config(**dict(ok, n_steps=10)).to_c()), ctypes.byref(nb)) == 2
    assert b"lightcone" in lib.pm_last_error()
    # the lightcone is seen along the line of sight: rsd_axis must be 3
    assert lib.pm_workspace_bytes(ctypes.byref(api.Config(**dict(ok, rsd_axis=2)).to_c()), ctypes.byref(nb)) == 1
    assert lib.pm_workspace_bytes(ctypes.byref(api.Config(**dict(ok, n_steps=18)).to_c()), ctypes.byref(nb)) == 0
    # the snapshots must be states after the initial condition
    assert lib.pm_workspace_bytes(ctypes.byref(api.Config(**dict(ok, a_init=0.8, n_steps=2)).to_c()),
                                  ctypes.byref(nb)) == 2


def test_host_power_table_matches_oracle(lib):
    from paper_2604_26823_gb300 import api
    lnk, lnp = api.pm_linear_power_table()
    rk, rp = C.linear_power_table()
    np.testing.assert_allclose(lnk, rk, rtol=0, atol=1e-13)
    np.testing.assert_allclose(lnp, rp, rtol=0, atol=1e-7)


def test_analysis_and_annealing_argument_checks_without_gpu(lib):
    """Argument errors of the plan-free entry points are reported before any
    device call."""
    z = ctypes.c_void_p(256)       # never dereferenced: the checks fail first
    # coarsening: factor must be a power of two dividing n
    assert lib.pm_coarsen(32, 3, 0, 0, z, z, None) == 1
    assert lib.pm_coarsen(32, 64, 0, 0, z, z, None) == 1
    assert lib.pm_coarsen(48, 2, 0, 0, z, z, None) == 1
    assert lib.pm_coarsen(32, 2, 7, 0, z, z, None) == 1
    assert lib.pm_coarsen(32, 2, 0, 2, z, z, None) == 1
    assert lib.pm_coarsen(32, 2, 0, 0, None, z, None) == 1
    # cosines / confusion: NULL arrays and bad precision
    assert lib.pm_eigvec_cosines(10, 0, None, z, z, None) == 1
    assert lib.pm_eigvec_cosines(10, 5, z, z, z, None) == 1
    assert lib.pm_eigvec_cosines(-1, 0, z, z, z, None) == 1
    assert lib.pm_confusion(10, 0, None, z, None, z, None) == 1
    assert lib.pm_confusion(10, 0, z, z, None, None, None) == 1
    # plan-bound entry points refuse a NULL plan
    assert lib.pm_refine_noise(None, z, 16, z, z, None) == 1
    assert lib.pm_tweb(None, z, 2.0, 0.16, z, None, None, None) == 1
    assert lib.pm_smooth(None, z, 2.0, z, None) == 1
    d = (ctypes.c_double * 4)()
    assert lib.pm_power_spectra(None, z, None, 4, 0.1, 1.0, d, None, None, d, None, None) == 1
    assert lib.pm_fma_rate(2, 100, z, d, None) == 1
    assert lib.pm_fma_rate(1, 0, z, d, None) == 1
    assert lib.pm_fma_rate(1, 100, None, d, None) == 1
    assert lib.pm_distance_table(0.3, 0.5, 1, d, d) == 1
    assert lib.pm_distance_table(0.3, 1.5, 4, d, d) == 1


def test_binding_refuses_dtypes_other_than_f32_f64():
    """The element size follows the dtype: anything but float32 / float64 is
    refused by the binding before the library is called (a float16 or int32
    vector read as doubles would be overrun)."""
    import torch
    from paper_2604_26823_gb300 import api
    with pytest.raises(TypeError):
        api.pm_project_noalloc(torch.zeros(16, dtype=torch.float16))
    with pytest.raises(TypeError):
        api.pm_project_noalloc(torch.zeros(16, dtype=torch.int32))
    with pytest.raises(TypeError):
        api.pm_coarsen(torch.zeros((4, 4, 4), dtype=torch.bfloat16), 2)
    with pytest.raises(TypeError):
        api.pm_eigvec_cosines(torch.zeros((3, 3, 2, 2, 2), dtype=torch.int32),
                              torch.zeros((3, 3, 2, 2, 2), dtype=torch.int32))
    with pytest.raises(TypeError):
        api.pm_axpy(0.5, torch.zeros(8, dtype=torch.float16), torch.zeros(8, dtype=torch.float16))
    with pytest.raises(TypeError):
        api.pm_confusion(torch.zeros(8, dtype=torch.int32), torch.zeros(8, dtype=torch.int32),
                         R=torch.zeros(8, dtype=torch.float16))


def test_lbfgs_workspace_holds_a_spare_pair_slot(lib):
    """m + 1 (s, y) slots: a new pair is written into the spare slot and
    enters the history only when accepted."""
    nb = ctypes.c_size_t()
    assert lib.lbfgs_workspace_bytes(1024, 4, 0, ctypes.byref(nb)) == 0
    vec = 1024 * 4
    assert nb.value >= 2 * 5 * vec + 2 * vec
