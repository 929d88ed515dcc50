"""ctypes binding of the FP64 CPU oracle (vl2_oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the benchmark's
CPU-baseline / reference leg.  The product path never imports this module.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "vl2_oracle.cpp")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liborc.so")

HLLE, HLLD, HLLE_ROE = 0, 1, 2
DC, PLM, PPM, PLM_CHAR, PPM_CHAR = 0, 1, 2, 3, 4
VL2, RK1, RK2, RK3 = 0, 1, 2, 3

_lib = None


def build(force=False):
    """Compile the oracle with value-safe flags (no FMA contraction, no reassociation)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.orc_mesh_new.restype = ctypes.c_void_p
        L.orc_mesh_new.argtypes = [ip, ip, dp, dp, ctypes.c_double, ctypes.c_int, ip, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_double]
        L.orc_set_scalars.argtypes = [ctypes.c_void_p, dp]
        L.orc_set_forcing.argtypes = [ctypes.c_void_p, dp]
        L.orc_get_scalars.argtypes = [ctypes.c_void_p, dp]
        L.orc_mesh_free.argtypes = [ctypes.c_void_p]
        L.orc_set_prims.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
        L.orc_get_cons.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
        L.orc_get_prims.argtypes = [ctypes.c_void_p, dp]
        L.orc_fill_ghosts.argtypes = [ctypes.c_void_p]
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_double]
        L.orc_new_dt.argtypes = [ctypes.c_void_p, ctypes.c_double]
        L.orc_new_dt.restype = ctypes.c_double
        L.orc_floor_count.argtypes = [ctypes.c_void_p]
        L.orc_floor_count.restype = ctypes.c_long
        L.orc_emf_mismatch_count.argtypes = [ctypes.c_void_p]
        L.orc_emf_mismatch_count.restype = ctypes.c_long
        L.orc_debug_fluxes.argtypes = [ctypes.c_void_p, ctypes.c_int, dp, dp, dp]
        L.orc_debug_emfs.argtypes = [ctypes.c_void_p, ctypes.c_int, dp, dp, dp]
        L.orc_divb_norm.argtypes = [ctypes.c_void_p]
        L.orc_divb_norm.restype = ctypes.c_double
        L.orc_totals.argtypes = [ctypes.c_void_p, dp]
        L.orc_set_cons.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
        L.orc_riemann.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_double, dp]
        L.orc_riemann_jacobian.argtypes = [ctypes.c_int, ctypes.c_longlong, dp, dp, dp, ctypes.c_double, dp]
        L.orc_physical_flux.argtypes = [dp, ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_fast_speed.argtypes = [ctypes.c_double] * 6
        L.orc_fast_speed.restype = ctypes.c_double
        L.orc_roe_fast_speed.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double, dp]
        L.orc_vanleer_slope.argtypes = [ctypes.c_double] * 3
        L.orc_vanleer_slope.restype = ctypes.c_double
        L.orc_ppm_edges.argtypes = [dp, dp]
        L.orc_mhd_eigensystem.argtypes = [dp, ctypes.c_double, ctypes.c_double, dp, dp, dp]
        L.orc_char_slope.argtypes = [dp, ctypes.c_double, ctypes.c_double, dp]
        L.orc_char_ppm_edges.argtypes = [dp, ctypes.c_double, ctypes.c_double, dp]
        L.orc_ppm_face.argtypes = [dp]
        L.orc_ppm_face.restype = ctypes.c_double
        L.orc_count_face_ops.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, ctypes.c_double,
                                         ctypes.POINTER(ctypes.c_longlong)]
        L.orc_ct_corner.argtypes = [dp, dp, dp, dp, dp]
        L.orc_tl_step.argtypes = [ip, ip, dp, dp, ctypes.c_double, ctypes.c_int, ip, ctypes.c_double,
                                  ctypes.c_double] + [dp] * 16
        L.orc_step_cons.argtypes = [ip, ip, dp, dp, ctypes.c_double, ctypes.c_int, ip, ctypes.c_double,
                                    ctypes.c_double] + [dp] * 8
        L.orc_ct_corner.restype = ctypes.c_double
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ------------------------------------------------------------------------------------------------
# pointwise functions
# ------------------------------------------------------------------------------------------------

def riemann(solver, wl, wr, bn, gamma):
    f = np.zeros(7)
    wl, wr = _c64(wl), _c64(wr)
    lib().orc_riemann(solver, _dp(wl), _dp(wr), float(bn), float(gamma), _dp(f))
    return f


def riemann_jacobian(solver, wl, wr, bn, gamma):
    """dF/d(w_L, w_R, b_n) for n interfaces: wl, wr (n, 7), bn (n,) -> (n, 7, 15), by dual numbers."""
    wl, wr = _c64(np.atleast_2d(wl)), _c64(np.atleast_2d(wr))
    bn = _c64(np.atleast_1d(bn))
    n = wl.shape[0]
    jac = np.zeros((n, 7, 15))
    lib().orc_riemann_jacobian(solver, n, _dp(wl), _dp(wr), _dp(bn), float(gamma), _dp(jac))
    return jac


def physical_flux(w, bn, gamma):
    w = _c64(w)
    u, f = np.zeros(7), np.zeros(7)
    lib().orc_physical_flux(_dp(w), float(bn), float(gamma), _dp(u), _dp(f))
    return u, f


def fast_speed(d, p, bn, bt1, bt2, gamma):
    return lib().orc_fast_speed(d, p, bn, bt1, bt2, gamma)


def roe_fast_speed(wl, wr, bn, gamma):
    """(u~, c~_f): Roe-averaged normal velocity and the fast speed of the MHD Roe matrix (Einfeldt's HLLE)."""
    out = np.zeros(2)
    wl, wr = _c64(wl), _c64(wr)
    lib().orc_roe_fast_speed(_dp(wl), _dp(wr), float(bn), float(gamma), _dp(out))
    return float(out[0]), float(out[1])


def vanleer_slope(qm, q0, qp):
    return lib().orc_vanleer_slope(qm, q0, qp)


def mhd_eigensystem(w, bn, gamma):
    """(R, L, lam) of the primitive MHD system at w = (rho, v_n, v_t1, v_t2, p, b_t1, b_t2) with normal field
    bn: columns of R are the right eigenvectors, L = R^-1, lam the eigenvalues (ascending)."""
    q = _c64(np.asarray(w, dtype=np.float64))
    R, L, lam = np.zeros((7, 7)), np.zeros((7, 7)), np.zeros(7)
    lib().orc_mhd_eigensystem(_dp(q), float(bn), float(gamma), _dp(R), _dp(L), _dp(lam))
    return R, L, lam


def char_slope(qm, q0, qp, bn, gamma):
    """Limited slope of the characteristic reconstruction of the cell q0 between qm and qp (7 each)."""
    q = _c64(np.concatenate([np.asarray(a, dtype=np.float64) for a in (qm, q0, qp)]))
    out = np.zeros(7)
    lib().orc_char_slope(_dp(q), float(bn), float(gamma), _dp(out))
    return out


def char_ppm_edges(q5, bn, gamma):
    """Characteristic PPM (lower, upper) edge values of the middle of five states q5[5][7], as a (7, 2) array."""
    q = _c64(np.asarray(q5, dtype=np.float64).reshape(35))
    out = np.zeros(14)
    lib().orc_char_ppm_edges(_dp(q), float(bn), float(gamma), _dp(out))
    return out.reshape(7, 2)


def ppm_edges(q5):
    """(left, right) PPM edge values of the middle cell of q5 = (q_{i-2}, ..., q_{i+2})."""
    q = _c64(np.asarray(q5, dtype=np.float64))
    out = np.zeros(2)
    lib().orc_ppm_edges(_dp(q), _dp(out))
    return float(out[0]), float(out[1])


def ppm_face(q4):
    """Limited fourth-order PPM face value between q4[1] and q4[2]."""
    q = _c64(np.asarray(q4, dtype=np.float64))
    return lib().orc_ppm_face(_dp(q))


def count_face_ops(recon, solver, q4, bn, gamma):
    """(add/sub, mul, div, sqrt, compare) FP64 operations of one face flux; q4 = states of cells
    i-2 .. i+1 in the sweep frame, shape (4, 7)."""
    q = _c64(q4).reshape(-1)
    out = (ctypes.c_longlong * 5)()
    lib().orc_count_face_ops(recon, solver, _dp(q), float(bn), float(gamma), out)
    return np.array(out[:], dtype=np.int64)


def ct_corner(ea, eb, ec, ma, mb):
    arrs = [_c64(a) for a in (ea, eb, ec, ma, mb)]
    return lib().orc_ct_corner(*[_dp(a) for a in arrs])


def _geom_args(nx, mb, xmin, xmax, bc):
    return ((ctypes.c_int * 3)(*nx), (ctypes.c_int * 3)(*mb), (ctypes.c_double * 3)(*xmin),
            (ctypes.c_double * 3)(*xmax), (ctypes.c_int * 6)(*bc))


def tl_step(prob_geom, dt, state, tangent, gamma=5.0 / 3.0, riemann=HLLD, ct_delta=0.0):
    """Tangent-linear of one VL2 cycle (dual numbers): state/tangent = (u, b1, b2, b3) global arrays.
    prob_geom = (nx, mb, xmin, xmax, bc); ct_delta > 0 takes the smoothed CT upwind weight, whose
    derivative in the mass flux the tangent carries.  Returns (new state, J @ tangent)."""
    nx, mb, xmin, xmax, bc = prob_geom
    ins = [_c64(a) for a in state] + [_c64(a) for a in tangent]
    outs = [np.zeros_like(a) for a in ins]
    g = _geom_args(nx, mb, xmin, xmax, bc)
    lib().orc_tl_step(g[0], g[1], g[2], g[3], float(gamma), riemann, g[4], float(dt), float(ct_delta),
                      *[_dp(a) for a in ins[:4]], *[_dp(a) for a in ins[4:]], *[_dp(a) for a in outs[:4]],
                      *[_dp(a) for a in outs[4:]])
    return tuple(outs[:4]), tuple(outs[4:])


def step_cons(prob_geom, dt, state, gamma=5.0 / 3.0, riemann=HLLD, ct_delta=0.0):
    """One VL2 cycle from a conserved state (global arrays); returns the new state."""
    nx, mb, xmin, xmax, bc = prob_geom
    ins = [_c64(a) for a in state]
    outs = [np.zeros_like(a) for a in ins]
    g = _geom_args(nx, mb, xmin, xmax, bc)
    lib().orc_step_cons(g[0], g[1], g[2], g[3], float(gamma), riemann, g[4], float(dt), float(ct_delta),
                        *[_dp(a) for a in ins],
                        *[_dp(a) for a in outs])
    return tuple(outs)


# ------------------------------------------------------------------------------------------------
# mesh
# ------------------------------------------------------------------------------------------------

class Mesh:
    """Oracle mesh of equal-size MeshBlocks holding one VL2 state.  recon is the reconstruction of the
    higher-order stages (PLM or PPM); ng the ghost layers (default 2, or 3 with PPM); nscalars the passive
    scalars (eq. passive_scalars); ct_delta > 0 smooths the CT upwind switch (an option, not the paper's)."""

    def __init__(self, nx, mb, xmin=(0.0, 0.0, 0.0), xmax=(1.0, 1.0, 1.0), gamma=5.0 / 3.0,
                 riemann=HLLD, bc=(0,) * 6, dfloor=1e-12, pfloor=1e-12, integrator=VL2, recon=PLM, ng=None,
                 nscalars=0, ct_delta=0.0):
        self.nx = tuple(int(v) for v in nx)
        self.mb = tuple(int(v) for v in mb)
        self.xmin, self.xmax = tuple(xmin), tuple(xmax)
        self.gamma = gamma
        L = lib()
        ia = (ctypes.c_int * 3)(*self.nx)
        ib = (ctypes.c_int * 3)(*self.mb)
        da = (ctypes.c_double * 3)(*self.xmin)
        db = (ctypes.c_double * 3)(*self.xmax)
        bcs = (ctypes.c_int * 6)(*bc)
        self.ng = (3 if recon in (PPM, PPM_CHAR) else 2) if ng is None else int(ng)
        self.nscalars = int(nscalars)
        self._h = L.orc_mesh_new(ia, ib, da, db, gamma, riemann, bcs, dfloor, pfloor, integrator, recon, self.ng,
                                 self.nscalars, float(ct_delta))
        if not self._h:
            raise ValueError("invalid oracle mesh parameters")

    @classmethod
    def from_problem(cls, prob, **kw):
        m = cls(prob.nx, kw.pop("mb", prob.mb), prob.xmin, prob.xmax, prob.gamma, bc=prob.bc, **kw)
        m.set_prims(prob.w, prob.b1, prob.b2, prob.b3)
        return m

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_mesh_free(h)
            self._h = None

    @property
    def shape(self):
        return (self.nx[2], self.nx[1], self.nx[0])

    @property
    def dx(self):
        return tuple((self.xmax[d] - self.xmin[d]) / self.nx[d] for d in range(3))

    def face_shapes(self):
        NX, NY, NZ = self.nx
        return (NZ, NY, NX + 1), (NZ, NY + 1, NX), (NZ + 1, NY, NX)

    def set_prims(self, w, b1, b2, b3):
        arrs = [_c64(a) for a in (w, b1, b2, b3)]
        lib().orc_set_prims(self._h, *[_dp(a) for a in arrs])

    def set_cons(self, u, b1, b2, b3):
        arrs = [_c64(a) for a in (u, b1, b2, b3)]
        lib().orc_set_cons(self._h, *[_dp(a) for a in arrs])

    def get_cons(self):
        u = np.zeros((5,) + self.shape)
        b = [np.zeros(s) for s in self.face_shapes()]
        lib().orc_get_cons(self._h, _dp(u), *[_dp(x) for x in b])
        return u, b[0], b[1], b[2]

    def set_scalars(self, c):
        """Concentrations c (nscalars, NZ, NY, NX); the state must be set first (rho C = rho c)."""
        c = _c64(np.asarray(c, dtype=np.float64).reshape((self.nscalars,) + self.shape))
        lib().orc_set_scalars(self._h, _dp(c))

    def set_forcing(self, a):
        """Forcing acceleration a (3, NZ, NY, NX) at the cell centres, or None to remove it."""
        if a is None:
            lib().orc_set_forcing(self._h, None)
            return
        self._acc = _c64(np.asarray(a, dtype=np.float64).reshape((3,) + self.shape))
        lib().orc_set_forcing(self._h, _dp(self._acc))

    def get_scalars(self):
        """Scalar masses rho C, (nscalars, NZ, NY, NX)."""
        out = np.zeros((self.nscalars,) + self.shape)
        lib().orc_get_scalars(self._h, _dp(out))
        return out

    def get_prims(self):
        w = np.zeros((8,) + self.shape)
        lib().orc_get_prims(self._h, _dp(w))
        return w

    def fill_ghosts(self):
        lib().orc_fill_ghosts(self._h)

    def step(self, dt):
        lib().orc_step(self._h, float(dt))

    def new_dt(self, cfl):
        return lib().orc_new_dt(self._h, float(cfl))

    def floor_count(self):
        return lib().orc_floor_count(self._h)

    def emf_mismatch_count(self):
        return lib().orc_emf_mismatch_count(self._h)

    def debug_fluxes(self, recon):
        NX, NY, NZ = self.nx
        fx = np.zeros((7, NZ, NY, NX + 1))
        fy = np.zeros((7, NZ, NY + 1, NX))
        fz = np.zeros((7, NZ + 1, NY, NX))
        lib().orc_debug_fluxes(self._h, recon, _dp(fx), _dp(fy), _dp(fz))
        return fx, fy, fz

    def debug_emfs(self, recon):
        NX, NY, NZ = self.nx
        e1 = np.zeros((NZ + 1, NY + 1, NX))
        e2 = np.zeros((NZ + 1, NY, NX + 1))
        e3 = np.zeros((NZ, NY + 1, NX + 1))
        lib().orc_debug_emfs(self._h, recon, _dp(e1), _dp(e2), _dp(e3))
        return e1, e2, e3

    def divb_norm(self):
        return lib().orc_divb_norm(self._h)

    def totals(self):
        out = np.zeros(8)
        lib().orc_totals(self._h, _dp(out))
        return out

    def run(self, t_end, cfl=0.3, max_steps=100000):
        """Advance to t_end with the CFL step, the last step clipped to land on t_end."""
        t, nsteps = 0.0, 0
        while t < t_end and nsteps < max_steps:
            dt = self.new_dt(cfl)
            if t + dt > t_end:
                dt = t_end - t
            self.step(dt)
            t += dt
            nsteps += 1
        return nsteps
