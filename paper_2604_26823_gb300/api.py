"""Python binding of the GB300 particle-mesh library (argument marshalling).

Every numerical step runs in the CUDA kernels behind the C ABI; PyTorch only
provides device memory (tensors, workspaces) and streams.  The functions keep
the C names (``pm_forward``, ``pm_adjoint``, ``lbfgs_step``,
``project_rank_match``, ...) and take ``Plan`` / ``LBFGS`` objects and CUDA
tensors.
"""
import ctypes
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib as L


def _stream(stream=None, device=None):
    """The given stream, else the current stream of ``device`` (of the current
    device when None)."""
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return ctypes.c_void_p(s.cuda_stream)


def _on(device):
    """Context that makes ``device`` current for one library call: kernels,
    the default stream and any per-device state of the library then belong to
    the device that holds the arguments."""
    return torch.cuda.device(device)


_PREC_OF = {torch.float32: L.PM_PREC_F32, torch.float64: L.PM_PREC_F64}


def _prec(t, name):
    """Library precision of a tensor; only float32 and float64 are accepted
    (any other dtype would be read with the wrong element size)."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype not in _PREC_OF:
        raise TypeError(f"{name} must be float32 or float64, not {t.dtype}")
    return _PREC_OF[t.dtype]


def _ptr(t, dtype, numel, name, device=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != numel:
        raise ValueError(f"{name} must be a contiguous {dtype} tensor with {numel} elements")
    if device is not None and t.device != torch.device(device):
        raise ValueError(f"{name} is on {t.device}, the call runs on {device}")
    return ctypes.c_void_p(t.data_ptr())


@dataclass
class Config:
    """Mirror of ``pm_config`` (Sec. 2.2.1 / 2.2.2 parameters)."""
    n: int
    box: float
    n_steps: int = 10
    lpt_order: int = 2
    rsd_axis: int = -1                # -1 none, 0..2 plane parallel, 3 radial from `observer`
    likelihood: str = "gaussian"      # "gaussian" | "poisson"
    bias: str = "auto"                # "auto" (gaussian: linear, poisson: power law) | "linear" | "powerlaw_sigmoid"
    precision: str = "f32"            # "f32" | "f64"
    checkpoint_every: int = 0
    omega_m: float = 0.25
    a_init: float = 0.1
    bias_b: float = 1.5
    sigma: float = 1.0
    alpha: float = 0.7
    delta_th: float = 1.2
    K: float = 3.0
    nbar_cell: float = 1.0
    rho_floor: float = 1e-3
    prior_weight: float = 1.0
    observer: tuple = (0.0, 0.0, 0.0)  # Mpc/h, box coordinates (rsd_axis = 3)
    lightcone: bool = False            # observe on the past light cone (needs rsd_axis = 3)

    def to_c(self):
        c = L.pm_config()
        c.n, c.n_steps, c.lpt_order, c.rsd_axis = self.n, self.n_steps, self.lpt_order, self.rsd_axis
        c.likelihood = {"gaussian": L.PM_LIK_GAUSSIAN, "poisson": L.PM_LIK_POISSON}[self.likelihood]
        c.bias = {"auto": L.PM_BIAS_AUTO, "linear": L.PM_BIAS_LINEAR,
                  "powerlaw_sigmoid": L.PM_BIAS_POWERLAW_SIGMOID}[self.bias]
        c.precision = {"f32": L.PM_PREC_F32, "f64": L.PM_PREC_F64}[self.precision]
        c.checkpoint_every = self.checkpoint_every
        c.lightcone = 1 if self.lightcone else 0
        for f in ("box", "omega_m", "a_init", "bias_b", "sigma", "alpha", "delta_th", "K",
                  "nbar_cell", "rho_floor", "prior_weight"):
            setattr(c, f, float(getattr(self, f)))
        for i in range(3):
            c.observer[i] = float(self.observer[i])
        return c

    @property
    def dtype(self):
        return torch.float32 if self.precision == "f32" else torch.float64


def pm_linear_power_table(omega_m=0.25, omega_b=0.045, h=0.73, sigma8=0.9, n_s=1.0,
                          k_min=1e-4, k_max=1e2, n_k=512):
    """Host table (ln k, ln P) of the no-wiggle LCDM P(k) (library host code)."""
    lib = L.load()
    lnk = np.zeros(n_k)
    lnp = np.zeros(n_k)
    L.check(lib.pm_linear_power_table(omega_m, omega_b, h, sigma8, n_s, k_min, k_max, n_k,
                                      lnk.ctypes.data_as(L._DP), lnp.ctypes.data_as(L._DP)),
            "pm_linear_power_table")
    return lnk, lnp


def pm_distance_table(omega_m, a_min=0.5, n=2049):
    """Host table (a_j, chi_j) of the lightcone's comoving distances (library host code)."""
    lib = L.load()
    a = np.zeros(n)
    chi = np.zeros(n)
    L.check(lib.pm_distance_table(omega_m, a_min, n, a.ctypes.data_as(L._DP), chi.ctypes.data_as(L._DP)),
            "pm_distance_table")
    return a, chi


def pm_growth(omega_m, a):
    lib = L.load()
    a = np.ascontiguousarray(a, dtype=np.float64)
    out = [np.zeros_like(a) for _ in range(4)]
    L.check(lib.pm_growth(omega_m, a.size, a.ctypes.data_as(L._DP),
                          *[o.ctypes.data_as(L._DP) for o in out]), "pm_growth")
    return dict(zip(("D1", "D2", "Gp1", "Gp2"), out))


class Plan:
    """A pm_plan plus its device workspace (a torch uint8 tensor)."""

    def __init__(self, config: Config, lnk=None, lnp=None, device="cuda"):
        lib = L.load()
        self.config = config
        self.cfg = config.to_c()
        self.n = config.n
        self.ncell = config.n ** 3
        self.dtype = config.dtype
        if lnk is None:
            lnk, lnp = pm_linear_power_table(omega_m=config.omega_m)
        lnk = np.ascontiguousarray(lnk, dtype=np.float64)
        lnp = np.ascontiguousarray(lnp, dtype=np.float64)
        nbytes = ctypes.c_size_t()
        L.check(lib.pm_workspace_bytes(ctypes.byref(self.cfg), ctypes.byref(nbytes)), "pm_workspace_bytes")
        self.workspace_bytes = nbytes.value
        self.workspace = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=device)
        self.device = self.workspace.device
        h = ctypes.c_void_p()
        with _on(self.device):
            L.check(lib.pm_plan_create(ctypes.byref(self.cfg), lnk.ctypes.data_as(L._DP),
                                       lnp.ctypes.data_as(L._DP), lnk.size,
                                       ctypes.c_void_p(self.workspace.data_ptr()), self.workspace_bytes,
                                       ctypes.byref(h)), "pm_plan_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            L.load().pm_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def mesh(self, t, name):
        return _ptr(t, self.dtype, self.ncell, name, self.device)

    def parts(self, t, name):
        return _ptr(t, self.dtype, 3 * self.ncell, name, self.device)

    def empty(self, *shape):
        return torch.empty(shape or (self.n, self.n, self.n), dtype=self.dtype, device=self.device)

    def call(self, fn, *args):
        """Run one C call with the plan's device current (its kernels and its
        default stream belong to that device)."""
        with _on(self.device):
            return getattr(L.load(), fn)(*args)


def pm_forward(plan, s, data, R, delta_out=None, stream=None):
    """loss = -log L + (w/2) sum s^2; optionally the final density contrast."""
    loss = ctypes.c_double()
    L.check(plan.call("pm_forward", plan.handle, plan.mesh(s, "s"), plan.mesh(data, "data"), plan.mesh(R, "R"),
                                ctypes.byref(loss), plan.mesh(delta_out, "delta_out"), _stream(stream, plan.device)),
            "pm_forward")
    return loss.value


def pm_adjoint(plan, s, data, R, loss_weight=1.0, cot_delta=None, grad_out=None, stream=None):
    """(loss, gradient of loss_weight * loss + <cot_delta, delta> wrt s)."""
    if grad_out is None:
        grad_out = torch.empty_like(s)
    loss = ctypes.c_double()
    L.check(plan.call("pm_adjoint", plan.handle, plan.mesh(s, "s"), plan.mesh(data, "data"), plan.mesh(R, "R"),
                                float(loss_weight), plan.mesh(cot_delta, "cot_delta"), ctypes.byref(loss),
                                plan.mesh(grad_out, "grad_out"), _stream(stream, plan.device)), "pm_adjoint")
    return loss.value, grad_out


def pm_last_terms(plan):
    a, b = ctypes.c_double(), ctypes.c_double()
    L.check(plan.call("pm_last_terms", plan.handle, ctypes.byref(a), ctypes.byref(b)), "pm_last_terms")
    return a.value, b.value


def pm_linear_field(plan, s, out=None, stream=None):
    out = plan.empty() if out is None else out
    L.check(plan.call("pm_linear_field", plan.handle, plan.mesh(s, "s"), plan.mesh(out, "out"), _stream(stream, plan.device)),
            "pm_linear_field")
    return out


def pm_lpt(plan, s, stream=None):
    disp, mom = plan.empty(3, plan.ncell), plan.empty(3, plan.ncell)
    L.check(plan.call("pm_lpt", plan.handle, plan.mesh(s, "s"), plan.parts(disp, "disp"), plan.parts(mom, "mom"),
                            _stream(stream, plan.device)), "pm_lpt")
    return disp, mom


def pm_force(plan, disp, with_density=False, stream=None):
    force = plan.empty(3, plan.ncell)
    dens = plan.empty() if with_density else None
    L.check(plan.call("pm_force", plan.handle, plan.parts(disp, "disp"), plan.parts(force, "force"),
                              plan.mesh(dens, "density"), _stream(stream, plan.device)), "pm_force")
    return (force, dens) if with_density else force


def pm_evolve(plan, s, stream=None):
    disp, mom = plan.empty(3, plan.ncell), plan.empty(3, plan.ncell)
    L.check(plan.call("pm_evolve", plan.handle, plan.mesh(s, "s"), plan.parts(disp, "disp"), plan.parts(mom, "mom"),
                               _stream(stream, plan.device)), "pm_evolve")
    return disp, mom


def pm_expected_counts(plan, s, R, out=None, stream=None):
    """Model mean per cell at s: the Poisson rate R nbar g(delta), or the
    Gaussian's biased field f(delta)."""
    out = plan.empty() if out is None else out
    L.check(plan.call("pm_expected_counts", plan.handle, plan.mesh(s, "s"), plan.mesh(R, "R"), plan.mesh(out, "out"),
                                        _stream(stream, plan.device)), "pm_expected_counts")
    return out


def pm_refine_noise(plan, s_coarse, fresh, out=None, stream=None):
    """White noise on the plan's mesh keeping the coarse field's modes (annealing)."""
    n_c = int(round(s_coarse.numel() ** (1.0 / 3.0)))
    out = plan.empty() if out is None else out
    L.check(plan.call("pm_refine_noise", plan.handle, _ptr(s_coarse, plan.dtype, n_c ** 3, "s_coarse"), n_c,
                                     plan.mesh(fresh, "fresh"), plan.mesh(out, "out"), _stream(stream, plan.device)),
            "pm_refine_noise")
    return out


def pm_coarsen(x, factor, mean=False, stream=None):
    """Block sums (mean=False) or means of factor^3 cells of a cubic CUDA mesh."""
    n = x.shape[0]
    nc = n // factor
    out = torch.empty((nc, nc, nc), dtype=x.dtype, device=x.device)
    prec = _prec(x, "x")
    with _on(x.device):
        L.check(L.load().pm_coarsen(n, factor, prec, 1 if mean else 0, _ptr(x, x.dtype, n ** 3, "x"),
                                    _ptr(out, x.dtype, nc ** 3, "out"), _stream(stream, x.device)), "pm_coarsen")
    return out


def pm_power_spectra(plan, a, b=None, n_bins=16, k_min=None, k_max=None, stream=None):
    """(k centres, P_aa, P_bb, P_ab, counts, r_c) as numpy arrays; default bins
    linear from the fundamental to the Nyquist wave number."""
    kf = 2 * np.pi / plan.config.box
    k_min = kf if k_min is None else k_min
    k_max = kf * plan.config.n / 2 if k_max is None else k_max
    out = [np.zeros(n_bins) for _ in range(5)]
    L.check(plan.call("pm_power_spectra", plan.handle, plan.mesh(a, "a"), plan.mesh(b, "b"), n_bins, k_min, k_max,
                      *[o.ctypes.data_as(L._DP) for o in out], _stream(stream, plan.device)),
            "pm_power_spectra")
    paa, pbb, pab, cnt, r = out
    edges = np.linspace(k_min, k_max, n_bins + 1)
    return 0.5 * (edges[1:] + edges[:-1]), paa, pbb, pab, cnt, r


def pm_smooth(plan, x, r_sm, out=None, stream=None):
    out = plan.empty() if out is None else out
    L.check(plan.call("pm_smooth", plan.handle, plan.mesh(x, "x"), float(r_sm), plan.mesh(out, "out"), _stream(stream, plan.device)),
            "pm_smooth")
    return out


def pm_tweb(plan, delta, r_sm=2.0, lambda_th=0.16, want_eig=True, want_evec=True, stream=None):
    """(labels int32 [n,n,n], eigenvalues [3,n,n,n] or None, eigenvectors
    [3 (which), 3 (component), n, n, n] or None)."""
    n = plan.config.n
    labels = torch.empty((n, n, n), dtype=torch.int32, device=plan.device)
    eig = torch.empty((3, n, n, n), dtype=plan.dtype, device=plan.device) if want_eig else None
    evec = torch.empty((3, 3, n, n, n), dtype=plan.dtype, device=plan.device) if want_evec else None
    L.check(plan.call("pm_tweb", plan.handle, plan.mesh(delta, "delta"), float(r_sm), float(lambda_th),
                             _ptr(labels, torch.int32, n ** 3, "labels"),
                             _ptr(eig, plan.dtype, 3 * n ** 3, "eig"), _ptr(evec, plan.dtype, 9 * n ** 3, "evec"),
                             _stream(stream, plan.device)), "pm_tweb")
    return labels, eig, evec


def pm_eigvec_cosines(va, vb, stream=None):
    """|e_i,a . e_i,b| per cell, [3, ...] for eigenvector fields [3, 3, ...]."""
    ncell = va.numel() // 9
    out = torch.empty((3,) + tuple(va.shape[2:]), dtype=va.dtype, device=va.device)
    prec = _prec(va, "va")
    dv = va.device
    with _on(dv):
        L.check(L.load().pm_eigvec_cosines(ncell, prec, _ptr(va, va.dtype, 9 * ncell, "va", dv),
                                           _ptr(vb, va.dtype, 9 * ncell, "vb", dv),
                                           _ptr(out, va.dtype, 3 * ncell, "out", dv), _stream(stream, dv)),
                "pm_eigvec_cosines")
    return out


def pm_confusion(labels_truth, labels_rec, R=None, stream=None):
    """4 x 4 numpy counts [truth, reconstructed] over the cells with R > 0."""
    ncell = labels_truth.numel()
    out = torch.empty(16, dtype=torch.int64, device=labels_truth.device)
    prec = _prec(R, "R") if R is not None else L.PM_PREC_F32
    dv = labels_truth.device
    with _on(dv):
        L.check(L.load().pm_confusion(ncell, prec, _ptr(labels_truth, torch.int32, ncell, "labels_truth", dv),
                                      _ptr(labels_rec, torch.int32, ncell, "labels_rec", dv),
                                      _ptr(R, R.dtype, ncell, "R", dv) if R is not None else None,
                                      _ptr(out, torch.int64, 16, "counts", dv), _stream(stream, dv)), "pm_confusion")
    return out.cpu().numpy().reshape(4, 4)


PROFILE_CLASSES = {"kdk": 0, "z_r2c": 1, "col": 2, "x_fused": 3, "z_c2r": 4, "adj_paint": 5,
                   "adj_gather": 6, "loss": 7}


def pm_profile(plan, enable=True, capacity=20000):
    L.check(plan.call("pm_profile", plan.handle, 1 if enable else 0, capacity if enable else 0), "pm_profile")


def pm_profile_read(plan, kernel_class):
    """(total milliseconds, launches, algorithmic bytes, implementation bytes,
    flops) of one kernel class since pm_profile."""
    c = PROFILE_CLASSES.get(kernel_class, kernel_class)
    ms, k = ctypes.c_double(), ctypes.c_int64()
    b, ib, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    L.check(plan.call("pm_profile_read", plan.handle, int(c), ctypes.byref(ms), ctypes.byref(k), ctypes.byref(b),
                      ctypes.byref(ib), ctypes.byref(fl)), "pm_profile_read")
    return ms.value, k.value, b.value, ib.value, fl.value


def pm_rom_fourier_counts(plan):
    out = np.zeros(100, dtype=np.int64)
    L.check(plan.call("pm_rom_fourier_counts", plan.handle, out.ctypes.data_as(L._I64P)), "pm_rom_fourier_counts")
    return out


def pm_count_positive(plan, R, stream=None):
    c = ctypes.c_int64()
    L.check(plan.call("pm_count_positive", plan.handle, plan.mesh(R, "R"), ctypes.byref(c), _stream(stream, plan.device)),
            "pm_count_positive")
    return c.value


def project_rank_match(plan, s_inout, mode, R=None, targets_real=None, targets_fourier=None, seed=0,
                       counter=0, stream=None, rank_out=None):
    """In place: Fourier matching, real-space matching, projection (by mode bits).
    Returns the number of reset values.  rank_out (optional int32 CUDA tensor
    of n^3 elements): with real-space matching, each cell's rank among the
    R > 0 cells before matching, -1 elsewhere."""
    nres = ctypes.c_int64()
    # the library reads exactly one target per matched value: refuse lists of
    # another length before the call
    tr = None
    if targets_real is not None and int(mode) & L.PM_ROM_REAL:
        need = pm_count_positive(plan, R, stream=stream)
        tr = _ptr(targets_real, plan.dtype, need, "targets_real", plan.device)
    tf = None
    if targets_fourier is not None and int(mode) & L.PM_ROM_FOURIER:
        need = int(pm_rom_fourier_counts(plan).sum())
        tf = _ptr(targets_fourier, plan.dtype, need, "targets_fourier", plan.device)
    rk = None if rank_out is None else _ptr(rank_out, torch.int32, plan.ncell, "rank_out", plan.device)
    L.check(plan.call("project_rank_match", plan.handle, plan.mesh(s_inout, "s"), int(mode),
                                        plan.mesh(R, "R") if R is not None else None, tr, tf,
                                        int(seed), int(counter), ctypes.byref(nres), rk,
                                        _stream(stream, plan.device)),
            "project_rank_match")
    return nres.value


def pm_project_noalloc(s_inout, seed=0, counter=0, stream=None):
    """Projection (z-score + reset) of a CUDA vector in place, with the
    library's static scratch instead of a workspace.  Returns the number of
    reset values."""
    prec = _prec(s_inout, "s")
    nres = ctypes.c_int64()
    dv = s_inout.device
    with _on(dv):   # the library looks up its static scratch on the current device
        L.check(L.load().pm_project_noalloc(s_inout.numel(), prec,
                                            _ptr(s_inout, s_inout.dtype, s_inout.numel(), "s", dv),
                                            int(seed), int(counter), ctypes.byref(nres), _stream(stream, dv)),
                "pm_project_noalloc")
    return nres.value


class LBFGS:
    """lbfgs_state plus its device workspace."""

    def __init__(self, n_elems, m=10, precision="f32", device="cuda"):
        lib = L.load()
        self.n = int(n_elems)
        self.prec = {"f32": L.PM_PREC_F32, "f64": L.PM_PREC_F64}[precision]
        self.dtype = torch.float32 if precision == "f32" else torch.float64
        nb = ctypes.c_size_t()
        L.check(lib.lbfgs_workspace_bytes(self.n, m, self.prec, ctypes.byref(nb)), "lbfgs_workspace_bytes")
        self.workspace = torch.empty(nb.value, dtype=torch.uint8, device=device)
        self.device = self.workspace.device
        h = ctypes.c_void_p()
        L.check(lib.lbfgs_create(self.n, m, self.prec, ctypes.c_void_p(self.workspace.data_ptr()), nb.value,
                                 ctypes.byref(h)), "lbfgs_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            L.load().lbfgs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lbfgs_reset(state):
    L.check(L.load().lbfgs_reset(state.handle), "lbfgs_reset")


def lbfgs_step(state, x_new, g_new, d_out=None, stream=None):
    """Push the pair from the previous point, then d = -H g.  Returns
    (d, g.d, |d|, pushed)."""
    if d_out is None:
        d_out = torch.empty_like(g_new)
    gd, dn, pushed = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    dv = state.device
    with _on(dv):
        L.check(L.load().lbfgs_step(state.handle, _ptr(x_new, state.dtype, state.n, "x_new", dv),
                                    _ptr(g_new, state.dtype, state.n, "g_new", dv),
                                    _ptr(d_out, state.dtype, state.n, "d", dv),
                                    ctypes.byref(gd), ctypes.byref(dn), ctypes.byref(pushed), _stream(stream, dv)),
                "lbfgs_step")
    return d_out, gd.value, dn.value, bool(pushed.value)


def pm_fma_rate(precision="f64", iters=4096, stream=None):
    """Measured FMA rate of the GPU in TFLOP/s (diagnostics)."""
    scratch = torch.empty(2, dtype=torch.float64, device="cuda")
    r = ctypes.c_double()
    with _on(scratch.device):
        L.check(L.load().pm_fma_rate(L.PM_PREC_F32 if precision == "f32" else L.PM_PREC_F64, int(iters),
                                     ctypes.c_void_p(scratch.data_ptr()), ctypes.byref(r),
                                     _stream(stream, scratch.device)), "pm_fma_rate")
    return r.value


def pm_axpy(alpha, x, y, out=None, stream=None):
    """out = y + alpha x (device kernel)."""
    if out is None:
        out = torch.empty_like(y)
    prec = _prec(y, "y")
    n = y.numel()
    dv = y.device
    with _on(dv):
        L.check(L.load().pm_axpy(n, prec, float(alpha), _ptr(x, y.dtype, n, "x", dv), _ptr(y, y.dtype, n, "y", dv),
                                 _ptr(out, y.dtype, n, "out", dv), _stream(stream, dv)), "pm_axpy")
    return out


class PMLoss(torch.autograd.Function):
    """loss(s) as an autograd node: forward runs pm_adjoint and caches the
    gradient, backward scales it by the incoming gradient."""

    @staticmethod
    def forward(ctx, s, plan, data, R):
        loss, grad = pm_adjoint(plan, s.detach().contiguous(), data, R)
        ctx.save_for_backward(grad)
        return torch.tensor(loss, dtype=torch.float64, device=s.device)

    @staticmethod
    def backward(ctx, gout):
        (grad,) = ctx.saved_tensors
        w = float(gout)
        # gout * grad = grad + (gout - 1) grad, by the library's axpy kernel
        out = grad if w == 1.0 else pm_axpy(w - 1.0, grad, grad)
        return out, None, None, None
