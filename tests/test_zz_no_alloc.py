"""The workspace-free projection entry point (for callers that cannot give
the library device memory, e.g. when all GPU memory belongs to another
allocator) must give the same result as the projection of
project_rank_match, call after call: its scratch is a static device array
that every call reuses, so a second call must not see the first call's
leftovers.  Collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_noalloc_projection_matches_plan_projection_twice(prec):
    from paper_2604_26823_gb300 import api, build, inputs
    build.build()
    n = 64
    dt = torch.float32 if prec == "f32" else torch.float64
    lnk, lnp = api.pm_linear_power_table()
    plan = api.Plan(api.Config(n=n, box=100.0, n_steps=1, precision=prec), lnk, lnp)
    s = (3.0 + 2.0 * inputs.white_noise(n, 1)).astype(np.float32)
    s.reshape(-1)[[7, 100, n ** 3 - 1]] = [300.0, -250.0, 280.0]
    a = torch.tensor(s, dtype=dt, device="cuda")     # existing entry point
    b = a.clone()                                     # workspace-free entry point
    tol = 1e-6 if prec == "f32" else 1e-12            # the projection tests' tolerance
    for call, counter in enumerate((11, 12)):
        na = api.project_rank_match(plan, a, api.L.PM_PROJECT, seed=6, counter=counter)
        nb = api.pm_project_noalloc(b, seed=6, counter=counter)
        assert na == nb == (3 if call == 0 else 0)
        np.testing.assert_allclose(b.cpu().numpy(), a.cpu().numpy(), rtol=tol, atol=tol)
    # NaN input or zero variance: an error, and the vector keeps its values
    bad = b.clone()
    bad.view(-1)[5] = float("nan")
    for vec in (bad, torch.full_like(b, 2.5)):
        before = vec.cpu().numpy().copy()
        with pytest.raises(api.L.PMError) as err:
            api.pm_project_noalloc(vec, seed=6, counter=13)
        assert err.value.status == api.L.PM_ERR_NONFINITE
        np.testing.assert_array_equal(vec.cpu().numpy(), before)
    # sizes beyond the static scratch are refused with a clear error
    lib = api.L.load()
    st = lib.pm_project_noalloc(2 ** 28 + 1, 0, api.ctypes.c_void_p(b.data_ptr()), 0, 0, None, None)
    assert st == 2 and b"exceeds the maximum" in lib.pm_last_error()
