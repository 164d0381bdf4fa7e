"""Context object over the C ABI.  Tensors must be CUDA tensors; outputs
are allocated with torch and filled by the library on the current stream."""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib
from ._lib import SphParams, SphStats, check


def default_params(**overrides) -> SphParams:
    lib = _lib.load()
    p = SphParams()
    lib.sph_default_params(C.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _f32(t, shape=None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("SPH tensors must live on the GPU")
    t = t.detach().to(torch.float32).contiguous()
    if shape is not None:
        t = t.reshape(shape)
    return t


def density_small_noalloc(pos, m, h_guess=None, box=1.0, n_ngb=48.0, max_iter=64):
    """Density + smoothing-length solve for one small box through the
    allocation-free entry point (direct summation, n <= 16384): the library
    allocates nothing; the output tensors below are allocated here by torch,
    on the caller's side of the interface.  Returns (h, rho, iterations)."""
    lib = _lib.load()
    pos = pos.detach().to(torch.float64).contiguous()
    m = _f32(m)
    hg = _f32(h_guess)
    n = pos.shape[0]
    h = torch.empty(n, device=pos.device, dtype=torch.float32)
    rho = torch.empty(n, device=pos.device, dtype=torch.float32)
    it = C.c_int32(0)
    check(lib.sph_density_small_noalloc(n, _ptr(pos), float(box), _ptr(m), _ptr(hg), float(n_ngb),
                                        int(max_iter), _ptr(h), _ptr(rho), C.byref(it), _stream()),
          "sph_density_small_noalloc")
    return h, rho, int(it.value)


class SPH:
    """One decomposition + state.  Typical use::

        s = SPH()
        s.build(pos)                 # (N, 3) float64, unit periodic box
        out = s.density(m)           # h, rho, omega
        acc, dudt = s.force(u, vel)
    """

    def __init__(self, **params):
        self.lib = _lib.load()
        self.params = default_params(**params)
        h = C.c_void_p()
        check(self.lib.sph_create(C.byref(self.params), C.byref(h)), "sph_create")
        self.h = h
        self.n = 0

    def close(self):
        if self.h:
            self.lib.sph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- build ---------------------------------------------------------------
    def build(self, pos, box=1.0, h_guess=None):
        pos = pos.detach().to(torch.float64).contiguous()
        hg = _f32(h_guess)
        self._keep = (pos, hg)
        self.n = pos.shape[0]
        check(self.lib.sph_build(self.h, self.n, _ptr(pos), float(box), _ptr(hg), _stream()),
              "sph_build")

    def build_batch(self, pos, offsets, boxes, h_guess=None):
        pos = pos.detach().to(torch.float64).contiguous()
        hg = _f32(h_guess)
        nbox = len(boxes)
        off = (C.c_int64 * (nbox + 1))(*[int(v) for v in offsets])
        bx = (C.c_double * nbox)(*[float(v) for v in boxes])
        self._keep = (pos, hg)
        self.n = pos.shape[0]
        check(self.lib.sph_build_batch(self.h, nbox, off, bx, _ptr(pos), _ptr(hg), _stream()),
              "sph_build_batch")

    # -- density -------------------------------------------------------------
    def density_fixed_h(self, m, h, count=False):
        m, h = _f32(m), _f32(h)
        z = lambda: torch.empty(self.n, device=m.device, dtype=torch.float32)
        rho, drho, nngb, dnngb = z(), z(), z(), z()
        cnt = torch.empty(self.n, device=m.device, dtype=torch.int32) if count else None
        check(self.lib.sph_density_fixed_h(self.h, _ptr(m), _ptr(h), _ptr(rho), _ptr(drho),
                                           _ptr(nngb), _ptr(dnngb), _ptr(cnt), _stream()),
              "sph_density_fixed_h")
        return dict(rho=rho, drho_dh=drho, nngb=nngb, dnngb_dh=dnngb, count=cnt)

    def density(self, m):
        m = _f32(m)
        z = lambda: torch.empty(self.n, device=m.device, dtype=torch.float32)
        h, rho, omega = z(), z(), z()
        it = C.c_int32(0)
        check(self.lib.sph_density(self.h, _ptr(m), _ptr(h), _ptr(rho), _ptr(omega),
                                   C.byref(it), _stream()), "sph_density")
        return dict(h=h, rho=rho, omega=omega, iters=int(it.value))

    # -- force ---------------------------------------------------------------
    def force(self, u, vel=None, count=False):
        u = _f32(u)
        vel = _f32(vel, (self.n, 3)) if vel is not None else None
        acc = torch.empty((self.n, 3), device=u.device, dtype=torch.float32)
        dudt = torch.empty(self.n, device=u.device, dtype=torch.float32)
        cnt = torch.empty(self.n, device=u.device, dtype=torch.int32) if count else None
        check(self.lib.sph_force(self.h, _ptr(u), _ptr(vel), _ptr(acc), _ptr(dudt), _ptr(cnt),
                                 _stream()), "sph_force")
        return acc, dudt, cnt

    def force_viscous(self, u, vel, alpha=0.8, c_cfl=0.25):
        """Force with the Monaghan-Balsara viscosity and the time step of
        Eq. (dt): returns (acc, dudt, dt, balsara).  No adjoint."""
        u = _f32(u)
        vel = _f32(vel, (self.n, 3))
        acc = torch.empty((self.n, 3), device=u.device, dtype=torch.float32)
        z = lambda: torch.empty(self.n, device=u.device, dtype=torch.float32)
        dudt, dt, f = z(), z(), z()
        check(self.lib.sph_force_viscous(self.h, _ptr(u), _ptr(vel), float(alpha), float(c_cfl),
                                         _ptr(acc), _ptr(dudt), _ptr(dt), _ptr(f), _stream()),
              "sph_force_viscous")
        return acc, dudt, dt, f

    # -- time integration -----------------------------------------------------
    def verlet_step(self, pos, vel, u, m, dt, box=1.0, alpha=0.8, c_cfl=0.25, slack=0.25):
        """One velocity-Verlet step (Section 4.1), in place on pos (N,3)
        float64, vel (N,3) float32 and u (N,) float32 device tensors (they
        must be contiguous of those dtypes).  Returns (dt_min, rebuilt): the
        smallest Eq. (dt) step at the end of the step and the number of
        decompositions built."""
        for t, dt_, shp in ((pos, torch.float64, 2), (vel, torch.float32, 2), (u, torch.float32, 1)):
            if t.dtype != dt_ or not t.is_contiguous() or not t.is_cuda or t.dim() != shp:
                raise ValueError("verlet_step updates pos/vel/u in place: contiguous CUDA tensors "
                                 "of dtype float64 / float32 / float32")
        m = _f32(m)
        n = pos.shape[0]
        dtm = C.c_float(0.0)
        nb = C.c_int32(0)
        check(self.lib.sph_verlet_step(self.h, n, _ptr(pos), _ptr(vel), _ptr(u), _ptr(m),
                                       float(box), float(dt), float(alpha), float(c_cfl),
                                       float(slack), C.byref(dtm), C.byref(nb), _stream()),
              "sph_verlet_step")
        self.n = n
        return float(dtm.value), int(nb.value)

    # -- adjoints ------------------------------------------------------------
    def force_adjoint(self, g_acc, g_dudt=None):
        g_acc = _f32(g_acc, (self.n, 3))
        g_dudt = _f32(g_dudt)
        dev = g_acc.device
        g_pos = torch.empty((self.n, 3), device=dev, dtype=torch.float32)
        z = lambda: torch.empty(self.n, device=dev, dtype=torch.float32)
        g_m, g_u, g_rho, g_drho, g_h = z(), z(), z(), z(), z()
        check(self.lib.sph_force_adjoint(self.h, _ptr(g_acc), _ptr(g_dudt), _ptr(g_pos), _ptr(g_m),
                                         _ptr(g_u), _ptr(g_rho), _ptr(g_drho), _ptr(g_h), _stream()),
              "sph_force_adjoint")
        return dict(g_pos=g_pos, g_m=g_m, g_u=g_u, g_rho=g_rho, g_drho=g_drho, g_h=g_h)

    def density_adjoint(self, g_rho, g_drho, g_h, g_pos, g_m):
        check(self.lib.sph_density_adjoint(self.h, _ptr(_f32(g_rho)), _ptr(_f32(g_drho)),
                                           _ptr(_f32(g_h)), _ptr(g_pos), _ptr(g_m), _stream()),
              "sph_density_adjoint")
        return g_pos, g_m

    def adjoint(self, g_rho=None, g_acc=None, g_dudt=None):
        dev = torch.device("cuda", torch.cuda.current_device())
        g_pos = torch.empty((self.n, 3), device=dev, dtype=torch.float32)
        g_m = torch.empty(self.n, device=dev, dtype=torch.float32)
        g_u = torch.empty(self.n, device=dev, dtype=torch.float32)
        check(self.lib.sph_adjoint(self.h, _ptr(_f32(g_rho)), _ptr(_f32(g_acc, (self.n, 3)) if g_acc is not None else None),
                                   _ptr(_f32(g_dudt)), _ptr(g_pos), _ptr(g_m), _ptr(g_u), _stream()),
              "sph_adjoint")
        return g_pos, g_m, g_u

    # -- introspection ---------------------------------------------------------
    def pairs(self, phase, cap=None):
        dev = torch.device("cuda", torch.cuda.current_device())
        cap = cap or max(1024, self.n * 128)
        pi = torch.empty(cap, device=dev, dtype=torch.int32)
        pj = torch.empty(cap, device=dev, dtype=torch.int32)
        n = C.c_int64(0)
        check(self.lib.sph_pairs_dump(self.h, int(phase), cap, _ptr(pi), _ptr(pj), C.byref(n),
                                      _stream()), "sph_pairs_dump")
        return pi[: n.value], pj[: n.value]

    def stats(self) -> dict:
        st = SphStats()
        check(self.lib.sph_get_stats(self.h, C.byref(st)), "sph_get_stats")
        d = {k: getattr(st, k) for k, _ in SphStats._fields_}
        d["top_level"] = list(st.top_level)[: max(1, min(8, st.nbox))]
        d["sweep_ms"] = list(st.sweep_ms)
        d["sweep_launches"] = list(st.sweep_launches)
        d["sweep_units"] = list(st.sweep_units)
        d["sweep_candidates"] = list(st.sweep_candidates)
        d["sweep_gathered"] = list(st.sweep_gathered)
        d["pairs_unlisted"] = st.pairs_unlisted
        d["pairs_unlisted_cut"] = st.pairs_unlisted_cut
        d["newton_active"] = list(st.newton_active)
        return d

    def set_sweep_config(self, warps_per_cta, sweep_cap, ctas_per_sm=0):
        check(self.lib.sph_set_sweep_config(self.h, int(warps_per_cta), int(sweep_cap),
                                            int(ctas_per_sm)), "sph_set_sweep_config")
        self.params.warps_per_cta = int(warps_per_cta)
        self.params.sweep_cap = int(sweep_cap)
        self.params.ctas_per_sm = int(ctas_per_sm)

    def profile(self, enable=True):
        check(self.lib.sph_profile(self.h, 1 if enable else 0), "sph_profile")

    def launch_count(self) -> int:
        return int(self.lib.sph_launch_count())

    def generation(self) -> int:
        """Counter of the forward state; changes with every build, density
        and force call on this context."""
        return int(self.lib.sph_state_generation(self.h))

    def sync_status(self):
        check(self.lib.sph_sync_status(self.h, _stream()), "sph_sync_status")
