"""GB300 implementation of the moving-magnet stray-field path of arXiv:1801.04181.

Python side of libmm (include/mm.h): `MovingMagnets` marshals torch tensors
(device memory, the current CUDA stream) into the C ABI.  Every step of the
computation runs in the CUDA kernels of the library; nothing here computes.
"""

import ctypes as C

import torch

from . import _native
from ._native import MMError, mm_options

__all__ = ["MovingMagnets", "MMError", "assign_lanes", "eval_kernel_fp64", "fft_plan", "load_library", "pair_context",
           "step_batch", "tuned_plan"]


def load_library():
    return _native.load()


def _check(lib, ctx, status):
    if status != 0:
        msg = lib.mm_last_error(ctx).decode() if ctx else ""
        raise MMError(status, msg)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _need_cuda_f32(t, shape=None):
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError("expected a contiguous float32 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("expected shape %s, got %s" % (shape, tuple(t.shape)))


class MovingMagnets:
    """Two magnets (0 base, 1 slider) and the slider's motion; one libmm context."""

    def __init__(self, margin=4, adaptive=True, rtol=1e-5, dt_min=1e-16, dt_max=1e-11, stream=None,
                 periodic=0, pbc_images=2, precision="fp32", integrator="rk45"):
        """periodic: 0 (open), or MM_PERIODIC_X | MM_PERIODIC_Y (1, 2, 3) with
        pbc_images periodic images on each side.  precision: "fp32", or
        "mixed" for the y transforms as split-BF16 tensor-core DFT products.
        integrator: "rk45" (Dormand-Prince 5(4)) or "euler" (explicit, fixed dt:
        needs adaptive=False)."""
        if precision not in ("fp32", "mixed"):
            raise ValueError("precision must be 'fp32' or 'mixed'")
        if integrator not in ("rk45", "euler"):
            raise ValueError("integrator must be 'rk45' or 'euler'")
        self.lib = _native.load()
        opt = mm_options()
        self.lib.mm_default_options(C.byref(opt))
        opt.precision = _native.MM_MIXED if precision == "mixed" else _native.MM_FP32
        opt.integrator = _native.MM_EULER if integrator == "euler" else _native.MM_RK45
        opt.periodic = int(periodic)
        opt.pbc_images = int(pbc_images)
        opt.margin = margin
        opt.adaptive = 1 if adaptive else 0
        opt.rtol = rtol
        opt.dt_min = dt_min
        opt.dt_max = dt_max
        if stream is None:
            stream = torch.cuda.current_stream()
        opt.stream = C.c_void_p(stream.cuda_stream)
        self.stream = stream
        ctx = C.c_void_p()
        _check(self.lib, None, self.lib.mm_create(C.byref(ctx), C.byref(opt)))
        self.ctx = ctx
        self.shapes = [None, None]

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.mm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self, status):
        _check(self.lib, self.ctx, status)

    def _in(self):
        """Order the context stream after the caller's stream (tensors it made)."""
        cur = torch.cuda.current_stream()
        if cur != self.stream:
            self.stream.wait_stream(cur)

    def _out(self, *ts):
        """Order the caller's stream after the context stream (tensors written there)."""
        cur = torch.cuda.current_stream()
        if cur != self.stream:
            cur.wait_stream(self.stream)
        return ts[0] if len(ts) == 1 else ts

    # ---------------------------------------------------------------- set-up
    def set_grid(self, mag, n, cell, offset=(0, 0, 0)):
        nx, ny, nz = n
        self._c(self.lib.mm_set_grid(self.ctx, mag, nx, ny, nz, *[float(c) for c in cell],
                                     _native._ll3(*[int(o) for o in offset])))
        self.shapes[mag] = (3, nz, ny, nx)

    def set_material(self, mag, Ms, Aex=0.0, Ku=0.0, ku_axis=(0.0, 0.0, 1.0), alpha=0.5):
        self._c(self.lib.mm_set_material(self.ctx, mag, Ms, Aex, Ku, _native._d3(*ku_axis), alpha))

    def set_external_field(self, H):
        self._c(self.lib.mm_set_external_field(self.ctx, _native._d3(*H)))

    def set_mechanics(self, mass, k, v_drive, gamma_v, direction=(1.0, 0.0, 0.0), x0_spring=0.0):
        self._c(self.lib.mm_set_mechanics(self.ctx, mass, k, v_drive, gamma_v, _native._d3(*direction),
                                          x0_spring))

    def set_magnetization(self, mag, m):
        _need_cuda_f32(m, self.shapes[mag])
        self._in()
        self._c(self.lib.mm_set_magnetization(self.ctx, mag, _ptr(m)))

    def get_magnetization(self, mag):
        out = torch.empty(self.shapes[mag], dtype=torch.float32, device="cuda")
        self._in()
        self._c(self.lib.mm_get_magnetization(self.ctx, mag, _ptr(out)))
        return self._out(out)

    def upload_magnetization(self, mag, m_host):
        if m_host.is_cuda or m_host.dtype != torch.float32 or not m_host.is_contiguous():
            raise ValueError("expected a contiguous float32 host tensor")
        self._c(self.lib.mm_upload_magnetization(self.ctx, mag, _ptr(m_host)))

    def download_magnetization(self, mag, out_host):
        if out_host.is_cuda or out_host.dtype != torch.float32 or not out_host.is_contiguous():
            raise ValueError("expected a contiguous float32 host tensor")
        self._c(self.lib.mm_download_magnetization(self.ctx, mag, _ptr(out_host)))
        return out_host

    def set_displacement(self, u_m):
        self._c(self.lib.mm_set_displacement(self.ctx, _native._d3(*u_m)))

    def set_slider_state(self, x, v, t):
        self._c(self.lib.mm_set_slider_state(self.ctx, x, v, t))

    def get_slider_state(self):
        x, v, t = C.c_double(), C.c_double(), C.c_double()
        self._c(self.lib.mm_get_slider_state(self.ctx, C.byref(x), C.byref(v), C.byref(t)))
        return x.value, v.value, t.value

    # ---------------------------------------------------------------- compute
    def compute_potential(self, src, prefiltered=False):
        dims = _native._i3()
        lo = _native._ll3()
        self._c(self.lib.mm_compute_potential(self.ctx, src, int(prefiltered), None, 0, dims, lo))
        out = torch.empty((dims[2], dims[1], dims[0]), dtype=torch.float32, device="cuda")
        self._in()
        self._c(self.lib.mm_compute_potential(self.ctx, src, int(prefiltered), _ptr(out), out.numel(),
                                              dims, lo))
        return self._out(out), (lo[0], lo[1], lo[2])

    def compute_stray_field(self, src):
        H = torch.empty(self.shapes[1 - src], dtype=torch.float32, device="cuda")
        self._in()
        self._c(self.lib.mm_compute_stray_field(self.ctx, src, _ptr(H)))
        return self._out(H)

    def compute_stray_field_fd4(self, src):
        """mm_compute_stray_field_fd4: the four-point difference variant of the stray field."""
        H = torch.empty(self.shapes[1 - src], dtype=torch.float32, device="cuda")
        self._in()
        self._c(self.lib.mm_compute_stray_field_fd4(self.ctx, src, _ptr(H)))
        return self._out(H)

    def compute_stray_field_componentwise(self, src):
        """mm_compute_stray_field_componentwise: the stray field by direct
        componentwise interpolation of the tensor field (comparison variant)."""
        H = torch.empty(self.shapes[1 - src], dtype=torch.float32, device="cuda")
        self._in()
        self._c(self.lib.mm_compute_stray_field_componentwise(self.ctx, src, _ptr(H)))
        return self._out(H)

    def eddy_field(self, mag, dBdt, sigma):
        """mm_eddy_field: (H_eddy (A/m), J (A/m^2), SOR sweeps) of magnet `mag`
        for the flux-density rate dBdt ((3, nz, ny, nx) float32 CUDA, T/s) and
        conductivity sigma (S/m)."""
        _need_cuda_f32(dBdt, self.shapes[mag])
        H = torch.empty(self.shapes[mag], dtype=torch.float32, device="cuda")
        J = torch.empty(self.shapes[mag], dtype=torch.float32, device="cuda")
        n = C.c_int()
        self._in()
        self._c(self.lib.mm_eddy_field(self.ctx, mag, _ptr(dBdt), float(sigma), _ptr(H), _ptr(J), C.byref(n)))
        self._out(H, J)
        return H, J, n.value

    def set_conductivity(self, mag, sigma):
        """mm_set_conductivity: couple the eddy field of magnet `mag` (sigma S/m) into the step."""
        self._c(self.lib.mm_set_conductivity(self.ctx, mag, float(sigma)))

    def eddy_field_on_other(self, mag, J):
        """mm_eddy_field_on_other: the field (A/m) of currents J ((3, nz, ny, nx)
        float32 CUDA, A/m^2) of magnet `mag` inside the other magnet."""
        _need_cuda_f32(J, self.shapes[mag])
        H = torch.empty(self.shapes[1 - mag], dtype=torch.float32, device="cuda")
        self._in()
        self._c(self.lib.mm_eddy_field_on_other(self.ctx, mag, _ptr(J), _ptr(H)))
        return self._out(H)

    def get_eddy_field(self, mag):
        """mm_get_eddy_field: the eddy field the next step adds for magnet `mag`."""
        H = torch.empty(self.shapes[mag], dtype=torch.float32, device="cuda")
        self._in()
        self._c(self.lib.mm_get_eddy_field(self.ctx, mag, _ptr(H)))
        return self._out(H)

    def compute_demag(self, mag):
        H = torch.empty(self.shapes[mag], dtype=torch.float32, device="cuda")
        self._in()
        self._c(self.lib.mm_compute_demag(self.ctx, mag, _ptr(H)))
        return self._out(H)

    def compute_fields(self):
        self._c(self.lib.mm_compute_fields(self.ctx))

    def get_force(self, on_mag):
        F = _native._d3()
        E = C.c_double()
        self._c(self.lib.mm_get_force(self.ctx, on_mag, F, C.byref(E)))
        return [F[0], F[1], F[2]], E.value

    def backward_energy(self, src, want_src=True, want_tgt=True):
        """Gradients of the energy of magnet 1 - src in the field of src:
        (dE/du (J/m, 3 floats), dE/dm_src (J, like m_src), dE/dm_tgt (J, like m_tgt))."""
        du = _native._d3()
        gs = torch.empty(self.shapes[src], dtype=torch.float32, device="cuda") if want_src else None
        gt = torch.empty(self.shapes[1 - src], dtype=torch.float32, device="cuda") if want_tgt else None
        self._in()
        self._c(self.lib.mm_backward_energy(self.ctx, src, du, _ptr(gs) if gs is not None else None,
                                            _ptr(gt) if gt is not None else None))
        self._out(gs)
        return [du[0], du[1], du[2]], gs, gt

    def compute_torque(self, mag):
        dm = torch.empty(self.shapes[mag], dtype=torch.float32, device="cuda")
        H = torch.empty(self.shapes[mag], dtype=torch.float32, device="cuda")
        self._in()
        self._c(self.lib.mm_compute_torque(self.ctx, mag, _ptr(dm), _ptr(H)))
        return self._out(dm, H)

    def step(self, nsteps, dt):
        t = C.c_double()
        d = C.c_double(dt)
        self._c(self.lib.mm_step(self.ctx, int(nsteps), C.byref(t), C.byref(d)))
        return t.value, d.value

    def power(self):
        """mm_get_power: dict with P_in, P_diss (one per magnet) and P_visc in W."""
        pin, pv = C.c_double(), C.c_double()
        pd = (C.c_double * 2)()
        self._c(self.lib.mm_get_power(self.ctx, C.byref(pin), pd, C.byref(pv)))
        return dict(P_in=pin.value, P_diss=[pd[0], pd[1]], P_visc=pv.value)

    def div_curl(self, H, cell):
        """mm_field_div_curl: (D, C), the mean |div H| and ||curl H|| (A/m^2) of a
        (3, nz, ny, nx) float32 CUDA field on cells `cell` (m)."""
        _need_cuda_f32(H)
        _, nz, ny, nx = H.shape
        D, Cc = C.c_double(), C.c_double()
        self._in()
        self._c(self.lib.mm_field_div_curl(self.ctx, _ptr(H), nx, ny, nz, *[float(c) for c in cell],
                                           C.byref(D), C.byref(Cc)))
        return D.value, Cc.value

    def step_stats(self):
        a, r = C.c_longlong(), C.c_longlong()
        self._c(self.lib.mm_get_step_stats(self.ctx, C.byref(a), C.byref(r)))
        return a.value, r.value

    def attempt_log(self, capacity=4096):
        """mm_get_attempt_log: the most recent step attempts, oldest first, as a
        list of dicts (t, dt, err, accepted)."""
        t = (C.c_double * capacity)()
        dt = (C.c_double * capacity)()
        err = (C.c_double * capacity)()
        acc = (C.c_int * capacity)()
        n = C.c_int()
        self._c(self.lib.mm_get_attempt_log(self.ctx, int(capacity), t, dt, err, acc, C.byref(n)))
        return [dict(t=t[i], dt=dt[i], err=err[i], accepted=bool(acc[i])) for i in range(n.value)]

    def clear_attempt_log(self):
        self._c(self.lib.mm_clear_attempt_log(self.ctx))

    def autotune(self, candidates=4, reps=3):
        """mm_autotune: time candidate FFT radix orders on this pair and keep the
        fastest per length (process-wide).  Returns the number of lengths timed."""
        n = C.c_int()
        self._c(self.lib.mm_autotune(self.ctx, int(candidates), int(reps), C.byref(n)))
        return n.value

    def get_state(self):
        n = C.c_size_t()
        self._c(self.lib.mm_get_state(self.ctx, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._c(self.lib.mm_get_state(self.ctx, buf, C.byref(n)))
        return buf.raw

    def set_state(self, blob):
        buf = C.create_string_buffer(blob, len(blob))
        self._c(self.lib.mm_set_state(self.ctx, buf, len(blob)))

    def plan_info(self, src):
        q = (C.c_int * 3)()
        b = _native._i3()
        lo = _native._ll3()
        cd = _native._i3()
        self._c(self.lib.mm_get_plan_info(self.ctx, src, q, b, lo, cd))
        return dict(fft=(q[0], q[1]), Qz=q[2], box=(b[0], b[1], b[2]), box_lo=(lo[0], lo[1], lo[2]),
                    coef=(cd[0], cd[1], cd[2]))

    # ---------------------------------------------------------------- timing
    def set_timing(self, on):
        self._c(self.lib.mm_set_timing(self.ctx, int(on)))

    def timing(self, cls):
        ms, n = C.c_double(), C.c_longlong()
        self._c(self.lib.mm_get_timing(self.ctx, cls, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def reset_timing(self):
        self._c(self.lib.mm_reset_timing(self.ctx))

    def launch_count(self):
        return self.lib.mm_launch_count(self.ctx)


def step_batch(pairs, nsteps, dts):
    """mm_step_batch: advance every MovingMagnets in `pairs` by nsteps accepted
    steps, each with its own adaptive dt (dts: one step size per pair).
    Returns (times, next step sizes) as lists."""
    n = len(pairs)
    if len(dts) != n:
        raise ValueError("one dt per pair")
    lib = _native.load()
    ctxs = (C.c_void_p * n)(*[p.ctx.value for p in pairs])
    t = (C.c_double * n)()
    d = (C.c_double * n)(*[float(x) for x in dts])
    bad = C.c_int(-1)
    s = lib.mm_step_batch(ctxs, n, int(nsteps), t, d, C.byref(bad))
    if s != 0:
        i = bad.value
        msg = lib.mm_last_error(pairs[i].ctx).decode() if 0 <= i < n else ""
        raise MMError(s, "pair %d: %s" % (i, msg))
    return list(t), list(d)


def fft_plan(L):
    """mm_fft_plan: the radices (first stage first) the FFT passes use for length L."""
    lib = _native.load()
    r = (C.c_int * 8)()
    n = C.c_int()
    s = lib.mm_fft_plan(int(L), r, C.byref(n))
    if s != 0:
        raise MMError(s, "mm_fft_plan")
    return [r[i] for i in range(n.value)]


def tuned_plan(L):
    """mm_get_tuned_plan: the autotuned radix order of length L, or None."""
    lib = _native.load()
    r = (C.c_int * 8)()
    n = C.c_int()
    s = lib.mm_get_tuned_plan(int(L), r, C.byref(n))
    if s != 0:
        return None
    return [r[i] for i in range(n.value)]


def assign_lanes(costs, nlanes):
    """mm_assign_lanes: longest-processing-time spread of pairs over nlanes streams."""
    lib = _native.load()
    n = len(costs)
    c = (C.c_double * n)(*[float(x) for x in costs])
    out = (C.c_int * n)()
    s = lib.mm_assign_lanes(c, n, int(nlanes), out)
    if s != 0:
        raise MMError(s, "mm_assign_lanes")
    return list(out)


def spline_field_noalloc(coef, coef_lo, pos0_nodes, m_target, cell, Ms, H_out, FE_out, stream=None):
    """mm_spline_field_noalloc: stray field / force / energy from a coefficient box, no allocation.

    coef: (bz, by, bx) float32 CUDA tensor of B-spline coefficients whose node
    [0, 0, 0] is source lattice node coef_lo; pos0_nodes: source-lattice
    position of target cell (0, 0, 0); m_target: (3, nz, ny, nx) float32 CUDA.
    H_out (3, nz, ny, nx) float32 (or None) and FE_out (4,) float64 are
    caller-provided CUDA tensors (FE_out = [Fx, Fy, Fz, E]); nothing is
    allocated here.  Every tensor must sit on one device; the call runs with
    that device current.
    """
    lib = _native.load()
    _need_cuda_f32(coef)
    _need_cuda_f32(m_target)
    if coef.dim() != 3:
        raise ValueError("coef must be a (bz, by, bx) tensor")
    if m_target.dim() != 4 or m_target.shape[0] != 3:
        raise ValueError("m_target must be a (3, nz, ny, nx) tensor")
    if H_out is not None:
        _need_cuda_f32(H_out, tuple(m_target.shape))
    if FE_out is None or not (FE_out.is_cuda and FE_out.dtype == torch.float64 and FE_out.numel() == 4
                              and FE_out.is_contiguous()):
        raise ValueError("FE_out must be a contiguous (4,) float64 CUDA tensor")
    dev = coef.device
    for t in (m_target, H_out, FE_out):
        if t is not None and t.device != dev:
            raise ValueError("coef, m_target, H_out and FE_out must be on one device")
    bz, by, bx = coef.shape
    _, nz, ny, nx = m_target.shape
    with torch.cuda.device(dev):
        st = stream if stream is not None else torch.cuda.current_stream(dev)
        s = lib.mm_spline_field_noalloc(_ptr(coef), _native._i3(bx, by, bz), _native._ll3(*coef_lo),
                                        _native._d3(*pos0_nodes), _ptr(m_target), nx, ny, nz,
                                        *[float(c) for c in cell], float(Ms), _ptr(H_out), _ptr(FE_out),
                                        C.c_void_p(st.cuda_stream))
    if s != 0:
        raise MMError(s, "mm_spline_field_noalloc")
    return H_out, FE_out


def eval_kernel_fp64(kind, offsets_m, cell):
    """S (kind 0) or N (kind 1) at target-minus-source offsets (n, 3) metres, FP64 on the GPU."""
    lib = _native.load()
    off = torch.as_tensor(offsets_m, dtype=torch.float64, device="cuda").contiguous()
    n = off.shape[0]
    out = torch.empty((n, 3 if kind == 0 else 6), dtype=torch.float64, device="cuda")
    st = lib.mm_eval_kernel_fp64(kind, n, _ptr(off), *[float(c) for c in cell], _ptr(out))
    if st != 0:
        raise MMError(st, "mm_eval_kernel_fp64")
    return out


class InteractionEnergy(torch.autograd.Function):
    """E(m_src, m_tgt, u): the interaction energy of magnet 1 - src in the stray
    field of src (J), differentiable in both unit magnetisations and in the
    slider displacement u (metres, a float64 tensor of 3).  The forward sets
    the context's state and evaluates; the backward returns the gradients that
    mm_backward_energy computed with it (the transposed path, in CUDA)."""

    @staticmethod
    def forward(ctx, mm, src, m_src, m_tgt, u):
        mm.set_magnetization(src, m_src.detach())
        mm.set_magnetization(1 - src, m_tgt.detach())
        mm.set_displacement(tuple(float(v) for v in u.detach().cpu()))
        du, gs, gt = mm.backward_energy(src)
        _, E = mm.get_force(1 - src)
        ctx.save_for_backward(gs, gt, torch.tensor(du, dtype=torch.float64))
        return torch.tensor(E, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gE):
        gs, gt, du = ctx.saved_tensors
        g = float(gE)
        return None, None, g * gs, g * gt, g * du.to(gE.device)


from .pairs import pair_context  # noqa: E402  (needs MovingMagnets above)
