"""Python binding of the C ABI in include/vl2mhd.h (argument marshalling only).

Every step of the method runs in the CUDA library libvl2mhd.so; this module only converts arguments.
PyTorch provides the device workspace and the stream.  There is no CPU fallback: if the compiled
library is missing, loading it raises.

The module-level functions carry the ABI's names (mesh_create, block_layout, set_prims, step,
fill_ghosts, new_dt, get_cons, get_prims, divb_norm, totals); `Mesh` bundles them as methods.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libvl2mhd.so")
# the value-safe parity build of the same sources (IEEE division and square root, no FMA contraction)
LIB_PATH_VALUE_SAFE = os.path.join(HERE, "_build", "libvl2mhd_vs.so")

VL2_OK, VL2_E_ARG, VL2_E_CUDA, VL2_E_NONPHYS, VL2_E_TIMEOUT, VL2_E_STATE, VL2_E_NOMEM = range(7)
HLLE, HLLD, HLLE_ROE = 0, 1, 2
PERIODIC, OUTFLOW = 0, 1
VL2, RK1, RK2, RK3 = 0, 1, 2, 3  # time integrators (vl2_params.integrator)
FP64, MIXED = 0, 1
HOST, DEVICE = 0, 1
DC, PLM, PPM, PLM_CHAR, PPM_CHAR = 0, 1, 2, 3, 4  # reconstructions (vl2_params.recon for the higher-order stages)

STATUS_NAMES = {0: "VL2_OK", 1: "VL2_E_ARG", 2: "VL2_E_CUDA", 3: "VL2_E_NONPHYS", 4: "VL2_E_TIMEOUT",
                5: "VL2_E_STATE", 6: "VL2_E_NOMEM"}


class VL2Error(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int * 3), ("mb", ctypes.c_int * 3), ("ng", ctypes.c_int),
                ("xmin", ctypes.c_double * 3), ("xmax", ctypes.c_double * 3), ("gamma", ctypes.c_double),
                ("cfl", ctypes.c_double), ("riemann", ctypes.c_int), ("precision", ctypes.c_int),
                ("bc", ctypes.c_int * 6), ("dfloor", ctypes.c_double), ("pfloor", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("adjoint", ctypes.c_int), ("integrator", ctypes.c_int),
                ("recon", ctypes.c_int), ("nscalars", ctypes.c_int), ("ct_delta", ctypes.c_double),
                ("forcing", ctypes.c_int)]


class Layout(ctypes.Structure):
    _fields_ = [("nblocks", ctypes.c_int), ("nb", ctypes.c_int * 3), ("mb", ctypes.c_int * 3), ("ng", ctypes.c_int),
                ("sx", ctypes.c_int), ("sy", ctypes.c_int), ("sz", ctypes.c_int),
                ("block_stride_vars", ctypes.c_longlong), ("block_loc", ctypes.POINTER(ctypes.c_int)),
                ("neighbor", ctypes.POINTER(ctypes.c_int)), ("u", ctypes.c_void_p), ("b", ctypes.c_void_p * 3)]


_libs = {}
EXPORTS = ["vl2_workspace_bytes", "vl2_mesh_create", "vl2_mesh_destroy", "vl2_block_layout", "vl2_set_prims",
           "vl2_fill_ghosts", "vl2_step", "vl2_new_dt", "vl2_get_cons", "vl2_get_prims", "vl2_divb_norm",
           "vl2_totals", "vl2_floor_count", "vl2_debug_fluxes", "vl2_debug_emfs", "vl2_profile",
           "vl2_profile_read", "vl2_launch_count", "vl2_totals_noalloc", "vl2_batch_workspace_bytes",
           "vl2_batch_create", "vl2_batch_destroy", "vl2_batch_autotune", "vl2_batch_step", "vl2_batch_run",
           "vl2_batch_launch_count", "vl2_batch_last_error", "vl2_set_cons", "vl2_step_vjp", "vl2_prims_vjp",
           "vl2_debug_riemann_vjp", "vl2_last_error", "vl2_set_scalars", "vl2_get_scalars", "vl2_debug_fp64_peak",
           "vl2_debug_arith", "vl2_set_forcing", "vl2_tape_bytes", "vl2_step_record", "vl2_step_vjp_recorded",
           "vl2_set_flux_shape", "vl2_get_flux_shape", "vl2_batch_flux_shape", "vl2_batch_set_flux_shape",
           "vl2_debug_wait_timeout", "vl2_set_prims_async", "vl2_step_cfl", "vl2_last_dt"]
NOALLOC_MAX_NZ = 4096
K_PRIM, K_GHOSTS, K_FLUX_DC, K_FLUX_PLM, K_EMF, K_UPDATE, K_FLUX_PPM, K_SCALARS, K_FLUX_HALO = range(9)
KERNEL_KINDS = {K_PRIM: "prim", K_GHOSTS: "ghosts", K_FLUX_DC: "flux_dc", K_FLUX_PLM: "flux_plm", K_EMF: "emf",
                K_UPDATE: "update", K_FLUX_PPM: "flux_ppm", K_SCALARS: "scalars", K_FLUX_HALO: "flux_halo"}


def load(path: str = LIB_PATH):
    """Load libvl2mhd.so, or another build of it such as the value-safe one (raises if it has not been built:
    there is no fallback path).  Each build is opened once, in its own symbol namespace."""
    path = os.path.abspath(path)
    if path in _libs:
        return _libs[path]
    if not os.path.exists(path):
        raise RuntimeError("%s not found; build it with paper_2005_06651_gb300.build.build()" % path)
    L = ctypes.CDLL(path)
    vp, dp, sz = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t
    L.vl2_workspace_bytes.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_size_t)]
    L.vl2_mesh_create.argtypes = [ctypes.POINTER(Params), vp, sz, ctypes.POINTER(ctypes.c_void_p)]
    L.vl2_mesh_destroy.argtypes = [vp]
    L.vl2_block_layout.argtypes = [vp, ctypes.POINTER(Layout)]
    L.vl2_set_prims.argtypes = [vp, dp, dp, dp, dp, ctypes.c_int]
    L.vl2_fill_ghosts.argtypes = [vp]
    L.vl2_step.argtypes = [vp, ctypes.c_double]
    L.vl2_new_dt.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.vl2_get_cons.argtypes = [vp, dp, dp, dp, dp, ctypes.c_int]
    L.vl2_get_prims.argtypes = [vp, dp, ctypes.c_int]
    L.vl2_divb_norm.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.vl2_totals.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.vl2_floor_count.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    L.vl2_debug_fluxes.argtypes = [vp, ctypes.c_int, dp, dp, dp, ctypes.c_int]
    L.vl2_debug_emfs.argtypes = [vp, ctypes.c_int, dp, dp, dp, ctypes.c_int]
    L.vl2_profile.argtypes = [vp, ctypes.c_int]
    L.vl2_profile_read.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                                   ctypes.POINTER(ctypes.c_longlong)]
    L.vl2_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    L.vl2_totals_noalloc.argtypes = [vp, vp, vp, vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                     vp, vp]
    L.vl2_set_cons.argtypes = [vp, dp, dp, dp, dp, ctypes.c_int]
    L.vl2_step_vjp.argtypes = [vp, ctypes.c_double] + [dp] * 8
    L.vl2_prims_vjp.argtypes = [vp, dp, dp, dp]
    L.vl2_debug_riemann_vjp.argtypes = [ctypes.c_int, ctypes.c_longlong, dp, dp, dp, dp, ctypes.c_double, dp, vp]
    L.vl2_debug_fp64_peak.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, dp, vp]
    L.vl2_debug_arith.argtypes = [ctypes.c_int, ctypes.c_longlong, dp, dp, vp]
    L.vl2_set_forcing.argtypes = [vp, dp, ctypes.c_int]
    L.vl2_tape_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.vl2_step_record.argtypes = [vp, ctypes.c_double, vp]
    L.vl2_step_vjp_recorded.argtypes = [vp, ctypes.c_double, vp] + [dp] * 8
    L.vl2_batch_workspace_bytes.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
    L.vl2_batch_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, vp, sz, ctypes.POINTER(ctypes.c_void_p)]
    L.vl2_batch_destroy.argtypes = [vp]
    L.vl2_batch_autotune.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.vl2_batch_step.argtypes = [vp, vp, ctypes.c_int]
    L.vl2_batch_run.argtypes = [vp, ctypes.c_int, vp]
    L.vl2_batch_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    ip = ctypes.POINTER(ctypes.c_int)
    L.vl2_set_flux_shape.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.vl2_get_flux_shape.argtypes = [vp, ip, ip, ip, ip]
    L.vl2_batch_flux_shape.argtypes = [vp, ip, ip, ip]
    L.vl2_batch_set_flux_shape.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.vl2_debug_wait_timeout.argtypes = [ctypes.c_int, dp, vp]
    L.vl2_set_prims_async.argtypes = [vp, dp, dp, dp, dp, ctypes.c_int]
    L.vl2_step_cfl.argtypes = [vp]
    L.vl2_last_dt.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.vl2_batch_last_error.argtypes = [vp]
    L.vl2_batch_last_error.restype = ctypes.c_char_p
    L.vl2_last_error.argtypes = [vp]
    L.vl2_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("vl2_last_error", "vl2_batch_last_error"):
            getattr(L, name).restype = ctypes.c_int
    _libs[path] = L
    return L


def _check(status, mesh_handle=None, allow=(), lib=None):
    if status != VL2_OK and status not in allow:
        msg = (lib or load()).vl2_last_error(mesh_handle)
        raise VL2Error(status, msg.decode() if msg else "")
    return status


def _ptr(a):
    """(pointer, where) for a numpy array or a torch tensor (CPU or CUDA), without copying."""
    if a is None:
        return None, HOST
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous float64")
        return a.ctypes.data, HOST
    import torch

    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("tensors must be contiguous float64")
        return a.data_ptr(), (DEVICE if a.is_cuda else HOST)
    raise TypeError("expected a numpy array or a torch tensor")


def _where_of(ptrs):
    wheres = {w for p, w in ptrs if p is not None}
    if len(wheres) > 1:
        raise ValueError("all buffers of one call must live on the same side (host or device)")
    return wheres.pop() if wheres else HOST


class Mesh:
    """A mesh of equal-size MeshBlocks on one CUDA device; all methods call the C ABI."""

    def __init__(self, nx, mb, xmin=(0.0, 0.0, 0.0), xmax=(1.0, 1.0, 1.0), gamma=5.0 / 3.0, cfl=0.3,
                 riemann=HLLD, bc=(PERIODIC,) * 6, dfloor=1e-12, pfloor=1e-12, precision=FP64, device=None,
                 stream=None, adjoint=False, integrator=VL2, recon=PLM, ng=None, nscalars=0, ct_delta=0.0,
                 value_safe=False, forcing=False):
        import torch

        L = load(LIB_PATH_VALUE_SAFE if value_safe else LIB_PATH)
        self._L = L
        self.value_safe = bool(value_safe)
        self.nx, self.mb = tuple(int(v) for v in nx), tuple(int(v) for v in mb)
        self.xmin, self.xmax = tuple(float(v) for v in xmin), tuple(float(v) for v in xmax)
        self.gamma, self.cfl = float(gamma), float(cfl)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        p = Params()
        p.nx[:] = self.nx
        p.mb[:] = self.mb
        p.ng = (3 if recon in (PPM, PPM_CHAR) else 2) if ng is None else int(ng)
        p.recon = int(recon)
        p.nscalars = int(nscalars)
        p.ct_delta = float(ct_delta)
        self.nscalars = int(nscalars)
        p.xmin[:] = self.xmin
        p.xmax[:] = self.xmax
        p.gamma, p.cfl = self.gamma, self.cfl
        p.riemann, p.precision = int(riemann), int(precision)
        p.bc[:] = tuple(int(v) for v in bc)
        p.dfloor, p.pfloor = float(dfloor), float(pfloor)
        p.stream = ctypes.c_void_p(stream.cuda_stream)
        p.adjoint = 1 if adjoint else 0
        p.forcing = 1 if forcing else 0
        p.integrator = int(integrator)
        self._params = p
        nbytes = ctypes.c_size_t()
        _check(L.vl2_workspace_bytes(ctypes.byref(p), ctypes.byref(nbytes)), lib=L)
        self.workspace_bytes = int(nbytes.value)
        self._ws = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8, device=self.device)
        base = self._ws.data_ptr()
        aligned = (base + 255) & ~255
        h = ctypes.c_void_p()
        _check(L.vl2_mesh_create(ctypes.byref(p), ctypes.c_void_p(aligned), ctypes.c_size_t(self.workspace_bytes),
                                 ctypes.byref(h)), lib=L)
        self._h = h

    @classmethod
    def from_problem(cls, prob, **kw):
        m = cls(prob.nx, kw.pop("mb", prob.mb), prob.xmin, prob.xmax, prob.gamma, bc=prob.bc, **kw)
        m.set_prims(prob.w, prob.b1, prob.b2, prob.b3)
        return m

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._L.vl2_mesh_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- shapes ----
    @property
    def shape(self):
        return (self.nx[2], self.nx[1], self.nx[0])

    def face_shapes(self):
        NX, NY, NZ = self.nx
        return (NZ, NY, NX + 1), (NZ, NY + 1, NX), (NZ + 1, NY, NX)

    @property
    def ncells(self):
        return self.nx[0] * self.nx[1] * self.nx[2]

    # ---- ABI calls ----
    def set_prims(self, w, b1, b2, b3):
        keep = [np.ascontiguousarray(x, dtype=np.float64) if isinstance(x, np.ndarray) else x for x in (w, b1, b2, b3)]
        ptrs = [_ptr(x) for x in keep]
        where = _where_of(ptrs)
        _check(self._L.vl2_set_prims(self._h, *[ctypes.c_void_p(p) for p, _ in ptrs], where), self._h, lib=self._L)

    def set_prims_async(self, w, b1, b2, b3):
        """vl2_set_prims_async: enqueue the state from primitives without waiting (CUDA tensors, or page-locked
        host tensors).  The inputs must stay untouched until the mesh's stream has consumed them."""
        ptrs = [_ptr(x) for x in (w, b1, b2, b3)]
        where = _where_of(ptrs)
        _check(self._L.vl2_set_prims_async(self._h, *[ctypes.c_void_p(p) for p, _ in ptrs], where), self._h,
               lib=self._L)

    def step_cfl(self):
        """vl2_step_cfl: one VL2 cycle with its CFL step formed and read on the device (no wait)."""
        _check(self._L.vl2_step_cfl(self._h), self._h, lib=self._L)

    def last_dt(self, allow_nonphys=False):
        """The step of the last step_cfl (waits; reports as new_dt does)."""
        out = ctypes.c_double()
        _check(self._L.vl2_last_dt(self._h, ctypes.byref(out)), self._h,
               allow=(VL2_E_NONPHYS,) if allow_nonphys else (), lib=self._L)
        return out.value

    def streamed_steps(self, host_in, host_out, nsteps):
        """nsteps repetitions of: host_in (page-locked w, b1, b2, b3) to the device, vl2_set_prims_async,
        vl2_step_cfl, vl2_get_cons into device buffers, and those to host_out (page-locked u, b1, b2, b3).  Two
        copy streams and double-buffered device staging let each step's copies run beside the neighbouring
        steps' cycles; events order every buffer's reuse.  Waits for the last step; returns its dt."""
        import torch

        dev = self.device
        main = self.stream
        cin, cout = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        din = [tuple(torch.empty(x.shape, dtype=torch.float64, device=dev) for x in host_in) for _ in range(2)]
        dout = [tuple(torch.empty(x.shape, dtype=torch.float64, device=dev) for x in host_out) for _ in range(2)]
        in_ready, in_free, out_ready, out_free = ([torch.cuda.Event() for _ in range(2)] for _ in range(4))

        def upload(i):
            cin.wait_event(in_free[i])  # the cycle that read this buffer has consumed it
            with torch.cuda.stream(cin):
                for d, h in zip(din[i], host_in):
                    d.copy_(h, non_blocking=True)
            in_ready[i].record(cin)

        upload(0)
        for k in range(nsteps):
            i = k % 2
            if k + 1 < nsteps:
                upload(1 - i)
            main.wait_event(in_ready[i])
            self.set_prims_async(*din[i])
            in_free[i].record(main)
            self.step_cfl()
            main.wait_event(out_free[i])  # the copy out of this buffer two steps ago has finished
            self.get_cons(dout[i])
            out_ready[i].record(main)
            cout.wait_event(out_ready[i])
            with torch.cuda.stream(cout):
                for h, d in zip(host_out, dout[i]):
                    h.copy_(d, non_blocking=True)
            out_free[i].record(cout)
        cout.synchronize()
        return self.last_dt(allow_nonphys=True)

    def set_scalars(self, c):
        """Concentrations c (nscalars, NZ, NY, NX), host array or CUDA tensor; set the state first."""
        keep = np.ascontiguousarray(c, dtype=np.float64) if isinstance(c, np.ndarray) else c
        ptr, where = _ptr(keep)
        _check(self._L.vl2_set_scalars(self._h, ctypes.c_void_p(ptr), where), self._h, lib=self._L)

    def get_scalars(self):
        """Scalar masses rho C, (nscalars, NZ, NY, NX)."""
        out = np.empty((self.nscalars,) + self.shape)
        _check(self._L.vl2_get_scalars(self._h, ctypes.c_void_p(out.ctypes.data), HOST), self._h, lib=self._L)
        return out

    def set_forcing(self, a):
        """Forcing acceleration a (3, NZ, NY, NX) at the cell centres (host array or CUDA tensor), or None to
        remove it; the mesh needs forcing=True."""
        if a is None:
            _check(self._L.vl2_set_forcing(self._h, None, HOST), self._h, lib=self._L)
            return
        keep = np.ascontiguousarray(a, dtype=np.float64) if isinstance(a, np.ndarray) else a
        ptr, where = _ptr(keep)
        _check(self._L.vl2_set_forcing(self._h, ctypes.c_void_p(ptr), where), self._h, lib=self._L)

    def set_cons(self, u, b1, b2, b3):
        keep = [np.ascontiguousarray(x, dtype=np.float64) if isinstance(x, np.ndarray) else x for x in (u, b1, b2, b3)]
        ptrs = [_ptr(x) for x in keep]
        where = _where_of(ptrs)
        _check(self._L.vl2_set_cons(self._h, *[ctypes.c_void_p(p) for p, _ in ptrs], where), self._h, lib=self._L)

    def step_vjp(self, dt, lam, out=None):
        """J^T lam for one cycle of step dt at the current state; lam/out = (u, b1, b2, b3) CUDA tensors."""
        import torch

        if out is None:
            out = tuple(torch.empty_like(t) for t in lam)
        for t in tuple(lam) + tuple(out):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                raise ValueError("step_vjp takes contiguous float64 CUDA tensors")
        _check(self._L.vl2_step_vjp(self._h, float(dt), *[ctypes.c_void_p(t.data_ptr()) for t in lam],
                                   *[ctypes.c_void_p(t.data_ptr()) for t in out]), self._h, lib=self._L)
        return out

    def tape_bytes(self):
        n = ctypes.c_size_t()
        _check(self._L.vl2_tape_bytes(self._h, ctypes.byref(n)), self._h, lib=self._L)
        return int(n.value)

    def new_tape(self):
        """A device buffer (uint8 tensor view, 256-byte aligned) that holds one recorded cycle."""
        import torch

        nbytes = self.tape_bytes()
        raw = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        off = (-raw.data_ptr()) % 256
        return raw[off:off + nbytes]

    def step_record(self, dt, tape):
        """One cycle like step(dt), keeping in `tape` (from new_tape) what its adjoint reads."""
        _check(self._L.vl2_step_record(self._h, float(dt), ctypes.c_void_p(tape.data_ptr())), self._h, lib=self._L)

    def step_vjp_recorded(self, dt, tape, lam, out=None):
        """J^T lam of the cycle recorded in `tape` (same dt); lam/out = (u, b1, b2, b3) CUDA tensors."""
        import torch

        if out is None:
            out = tuple(torch.empty_like(t) for t in lam)
        for t in tuple(lam) + tuple(out):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                raise ValueError("step_vjp_recorded takes contiguous float64 CUDA tensors")
        _check(self._L.vl2_step_vjp_recorded(self._h, float(dt), ctypes.c_void_p(tape.data_ptr()),
                                             *[ctypes.c_void_p(t.data_ptr()) for t in lam],
                                             *[ctypes.c_void_p(t.data_ptr()) for t in out]), self._h, lib=self._L)
        return out

    def prims_vjp(self, w, lam_u, out=None):
        import torch

        if out is None:
            out = torch.empty_like(lam_u)
        _check(self._L.vl2_prims_vjp(self._h, ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(lam_u.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr())), self._h, lib=self._L)
        return out

    def fill_ghosts(self):
        _check(self._L.vl2_fill_ghosts(self._h), self._h, lib=self._L)

    def step(self, dt):
        _check(self._L.vl2_step(self._h, float(dt)), self._h, lib=self._L)

    def new_dt(self, allow_nonphys=False):
        out = ctypes.c_double()
        _check(self._L.vl2_new_dt(self._h, ctypes.byref(out)), self._h, allow=(VL2_E_NONPHYS,) if allow_nonphys else (),
               lib=self._L)
        return out.value

    def get_cons(self, out=None):
        """Conserved state (u, b1, b2, b3); into `out` (numpy or torch, host or device) or new numpy arrays."""
        if out is None:
            out = (np.empty((5,) + self.shape), *[np.empty(s) for s in self.face_shapes()])
        ptrs = [_ptr(x) for x in out]
        where = _where_of(ptrs)
        _check(self._L.vl2_get_cons(self._h, *[ctypes.c_void_p(p) if p else None for p, _ in ptrs], where), self._h, lib=self._L)
        return out

    def get_prims(self, out=None):
        if out is None:
            out = np.empty((8,) + self.shape)
        p, where = _ptr(out)
        _check(self._L.vl2_get_prims(self._h, ctypes.c_void_p(p), where), self._h, lib=self._L)
        return out

    def divb_norm(self):
        out = ctypes.c_double()
        _check(self._L.vl2_divb_norm(self._h, ctypes.byref(out)), self._h, lib=self._L)
        return out.value

    def totals(self):
        out = (ctypes.c_double * 8)()
        _check(self._L.vl2_totals(self._h, out), self._h, lib=self._L)
        return np.array(out[:])

    def floor_count(self):
        out = ctypes.c_longlong()
        _check(self._L.vl2_floor_count(self._h, ctypes.byref(out)), self._h, lib=self._L)
        return out.value

    def block_layout(self):
        lay = Layout()
        _check(self._L.vl2_block_layout(self._h, ctypes.byref(lay)), self._h, lib=self._L)
        n = lay.nblocks
        return {"nblocks": n, "nb": tuple(lay.nb), "mb": tuple(lay.mb), "ng": lay.ng,
                "strides": (lay.sx, lay.sy, lay.sz), "block_stride_vars": lay.block_stride_vars,
                "block_loc": np.ctypeslib.as_array(lay.block_loc, shape=(n, 3)).copy(),
                "neighbor": np.ctypeslib.as_array(lay.neighbor, shape=(n, 27)).copy(),
                "u": lay.u, "b": tuple(lay.b)}

    def profile(self, enable=True):
        _check(self._L.vl2_profile(self._h, int(bool(enable))), self._h, lib=self._L)

    def profile_read(self):
        """{kind: (ms, launches, units)} accumulated since the last read (resets)."""
        out = {}
        for k, name in KERNEL_KINDS.items():
            ms, n, u = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_longlong()
            _check(self._L.vl2_profile_read(self._h, k, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(u)), self._h, lib=self._L)
            out[name] = (ms.value, n.value, u.value)
        return out

    def launch_count(self):
        n = ctypes.c_longlong()
        _check(self._L.vl2_launch_count(self._h, ctypes.byref(n)), self._h, lib=self._L)
        return n.value

    def set_flux_shape(self, dc_threads=128, plm_lines=16, tma=0):
        """Launch shapes of the flux sweeps (vl2_set_flux_shape); no result bit depends on them."""
        _check(self._L.vl2_set_flux_shape(self._h, int(dc_threads), int(plm_lines), int(tma)), self._h, lib=self._L)

    def flux_shape(self):
        """(dc_threads, plm_lines, tma, tma_active) of this mesh (vl2_get_flux_shape)."""
        v = [ctypes.c_int() for _ in range(4)]
        _check(self._L.vl2_get_flux_shape(self._h, *[ctypes.byref(x) for x in v]), self._h, lib=self._L)
        return tuple(x.value for x in v)

    def debug_fluxes(self, recon):
        NX, NY, NZ = self.nx
        fx, fy, fz = np.empty((7, NZ, NY, NX + 1)), np.empty((7, NZ, NY + 1, NX)), np.empty((7, NZ + 1, NY, NX))
        _check(self._L.vl2_debug_fluxes(self._h, int(recon), *[ctypes.c_void_p(a.ctypes.data) for a in (fx, fy, fz)],
                                       HOST), self._h, lib=self._L)
        return fx, fy, fz

    def debug_emfs(self, recon):
        NX, NY, NZ = self.nx
        e1, e2, e3 = np.empty((NZ + 1, NY + 1, NX)), np.empty((NZ + 1, NY, NX + 1)), np.empty((NZ, NY + 1, NX + 1))
        _check(self._L.vl2_debug_emfs(self._h, int(recon), *[ctypes.c_void_p(a.ctypes.data) for a in (e1, e2, e3)],
                                     HOST), self._h, lib=self._L)
        return e1, e2, e3

    def run(self, t_end, max_steps=1_000_000):
        """Advance to t_end with the CFL step; the last step is clipped to land on t_end."""
        t, n = 0.0, 0
        while t < t_end and n < max_steps:
            dt = self.new_dt()
            if t + dt > t_end:
                dt = t_end - t
            self.step(dt)
            t += dt
            n += 1
        return n


def _noalloc_args(u, b1, b2, b3, out):
    """Validate the tensors of totals_noalloc before anything reaches the device: shapes first (u [5][NZ][NY][NX],
    b1 (NZ, NY, NX+1), b2 (NZ, NY+1, NX), b3 (NZ+1, NY, NX), out at least 8 elements), then contiguous
    float64 CUDA tensors on one device.  Returns (NX, NY, NZ)."""
    import torch

    for name, t in (("u", u), ("b1", b1), ("b2", b2), ("b3", b3), ("out", out)):
        if not isinstance(t, torch.Tensor):
            raise ValueError("totals_noalloc: %s must be a torch tensor" % name)
    if u.dim() != 4 or u.shape[0] != 5:
        raise ValueError("totals_noalloc: u must have shape (5, NZ, NY, NX), got %s" % (tuple(u.shape),))
    nz, ny, nx = (int(v) for v in u.shape[1:])
    want = {"b1": (nz, ny, nx + 1), "b2": (nz, ny + 1, nx), "b3": (nz + 1, ny, nx)}
    for name, t in (("b1", b1), ("b2", b2), ("b3", b3)):
        if tuple(t.shape) != want[name]:
            raise ValueError("totals_noalloc: %s must have shape %s, got %s" % (name, want[name], tuple(t.shape)))
    if out.numel() < 8:
        raise ValueError("totals_noalloc: out must hold at least 8 doubles")
    for name, t in (("u", u), ("b1", b1), ("b2", b2), ("b3", b3), ("out", out)):
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise ValueError("totals_noalloc: %s must be a contiguous float64 CUDA tensor" % name)
    if len({t.device for t in (u, b1, b2, b3, out)}) != 1:
        raise ValueError("totals_noalloc: all tensors must be on one device")
    return nx, ny, nz


def totals_noalloc(u, b1, b2, b3, dx, out, stream=None):
    """vl2_totals_noalloc on device tensors u [5][NZ][NY][NX], b1, b2, b3 (global layout) into the device
    tensor out (8 doubles), enqueued on `stream` (default: the current torch stream of u's device), with u's
    device current.  Allocates nothing."""
    import torch

    nx, ny, nz = _noalloc_args(u, b1, b2, b3, out)
    dims = (ctypes.c_int * 3)(nx, ny, nz)
    h = (ctypes.c_double * 3)(*dx)
    with torch.cuda.device(u.device):
        st = (stream or torch.cuda.current_stream(u.device)).cuda_stream
        _check(load().vl2_totals_noalloc(*[ctypes.c_void_p(t.data_ptr()) for t in (u, b1, b2, b3)], dims, h,
                                         ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st)))
    return out


def debug_riemann_vjp(riemann, wl, wr, bn, lf, gamma, stream=None):
    """vl2_debug_riemann_vjp on contiguous float64 CUDA tensors wl, wr, lf [n][7] and bn [n]: returns the
    [n][15] tensor lf . dF/d(w_L, w_R, b_n)."""
    import torch

    for t in (wl, wr, bn, lf):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise ValueError("debug_riemann_vjp takes contiguous float64 CUDA tensors")
    n = bn.shape[0]
    out = torch.empty((n, 15), dtype=torch.float64, device=bn.device)
    st = (stream or torch.cuda.current_stream(bn.device)).cuda_stream
    _check(load().vl2_debug_riemann_vjp(int(riemann), n, *[ctypes.c_void_p(t.data_ptr()) for t in (wl, wr, bn, lf)],
                                        float(gamma), ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st)))
    return out


AR_RCP_NR, AR_RSQRT_NR, AR_SQRT_NR, AR_INV_ANY, AR_ROOT_ANY, AR_RROOT_ANY, AR_TO_F32, AR_TO_F64, AR_IEEE_RCP, \
    AR_IEEE_SQRT, AR_CUDA_RSQRT, AR_CUDA_D2F = range(12)


def debug_arith(fn, x, stream=None):
    """vl2_debug_arith on a contiguous float64 CUDA tensor x: returns fn(x) as a new float64 tensor."""
    import torch

    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
        raise ValueError("debug_arith takes a contiguous float64 CUDA tensor")
    out = torch.empty_like(x)
    with torch.cuda.device(x.device):
        st = (stream or torch.cuda.current_stream(x.device)).cuda_stream
        _check(load().vl2_debug_arith(int(fn), x.numel(), ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st)))
    return out


def debug_wait_timeout(polls=1000, device=None):
    """vl2_debug_wait_timeout: 1 when the bounded wait on a phase that nothing completes gave up (expected)."""
    import torch

    dev = torch.device("cuda") if device is None else torch.device(device)
    with torch.cuda.device(dev):
        out = torch.full((1,), -1, dtype=torch.int32, device=dev)
        st = torch.cuda.current_stream(dev)
        _check(load().vl2_debug_wait_timeout(int(polls), ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st.cuda_stream)))
        return int(out.item())


def fp64_peak(device=None, iters=1 << 16, ctas=None, threads=256, repeats=5):
    """Measured FP64 peak (TFLOP/s): the best of `repeats` event-timed launches of vl2_debug_fp64_peak, each
    2 * 16 * iters * ctas * threads FP64 operations (fused multiply-adds count 2).  ctas defaults to 8 per SM."""
    import torch

    dev = torch.device("cuda") if device is None else torch.device(device)
    with torch.cuda.device(dev):
        props = torch.cuda.get_device_properties(dev)
        ctas = ctas or 8 * props.multi_processor_count
        out = torch.zeros(1, dtype=torch.float64, device=dev)
        st = torch.cuda.current_stream(dev)
        L = load()
        _check(L.vl2_debug_fp64_peak(int(iters) // 16, int(ctas), int(threads), ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(st.cuda_stream)))  # warm-up
        best = None
        for _ in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            _check(L.vl2_debug_fp64_peak(int(iters), int(ctas), int(threads), ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(st.cuda_stream)))
            e1.record(st)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
    flops = 2.0 * 16 * iters * ctas * threads
    return {"tflops": flops / (best / 1e3) / 1e12, "ms": best, "flops": flops, "ctas": ctas, "threads": threads}


def _bcheck(status, handle=None, lib=None):
    if status != VL2_OK:
        msg = (lib or load()).vl2_batch_last_error(handle)
        raise VL2Error(status, msg.decode() if msg else "")
    return status


class Batch:
    """Many independent meshes advanced together (vl2_batch_*).  Keeps the meshes alive."""

    def __init__(self, meshes):
        import torch

        self.meshes = list(meshes)
        if len({m._L._name for m in self.meshes}) > 1:
            raise ValueError("the meshes of a batch must come from one build of the library")
        L = self._L = self.meshes[0]._L
        arr = (ctypes.c_void_p * len(self.meshes))(*[m._h.value for m in self.meshes])
        self._arr = arr
        nbytes = ctypes.c_size_t()
        _bcheck(L.vl2_batch_workspace_bytes(arr, len(self.meshes), ctypes.byref(nbytes)), lib=L)
        dev = self.meshes[0].device
        self._ws = torch.empty(int(nbytes.value) + 256, dtype=torch.uint8, device=dev)
        aligned = (self._ws.data_ptr() + 255) & ~255
        h = ctypes.c_void_p()
        _bcheck(L.vl2_batch_create(arr, len(self.meshes), ctypes.c_void_p(aligned), nbytes, ctypes.byref(h)), lib=L)
        self._h = h

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._L.vl2_batch_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def ncells(self):
        return sum(m.ncells for m in self.meshes)

    def autotune(self):
        dc, pl = ctypes.c_int(), ctypes.c_int()
        _bcheck(self._L.vl2_batch_autotune(self._h, ctypes.byref(dc), ctypes.byref(pl)), self._h, lib=self._L)
        return dc.value, pl.value

    def step(self, dt):
        """One cycle with per-box steps dt (sequence of floats, or a CUDA float64 tensor)."""
        if isinstance(dt, np.ndarray) or isinstance(dt, (list, tuple)):
            a = np.ascontiguousarray(dt, dtype=np.float64)
            _bcheck(self._L.vl2_batch_step(self._h, ctypes.c_void_p(a.ctypes.data), HOST), self._h, lib=self._L)
        else:
            p, where = _ptr(dt)
            _bcheck(self._L.vl2_batch_step(self._h, ctypes.c_void_p(p), where), self._h, lib=self._L)

    def run(self, nsteps, want_dt=True):
        """nsteps cycles with per-box CFL steps formed on the device, as one graph launch."""
        out = np.empty(len(self.meshes)) if want_dt else None
        _bcheck(self._L.vl2_batch_run(self._h, int(nsteps), ctypes.c_void_p(out.ctypes.data) if want_dt else None),
                self._h, lib=self._L)
        return out

    def launch_count(self):
        n = ctypes.c_longlong()
        _bcheck(self._L.vl2_batch_launch_count(self._h, ctypes.byref(n)), self._h, lib=self._L)
        return n.value

    def set_flux_shape(self, dc_threads=128, plm_lines=16, tma=0):
        """Launch shapes of the batch's flux sweeps (vl2_batch_set_flux_shape)."""
        _bcheck(self._L.vl2_batch_set_flux_shape(self._h, int(dc_threads), int(plm_lines), int(tma)), self._h,
                lib=self._L)

    def flux_shape(self):
        """(dc_threads, plm_lines, tma) the batch's flux launches use (vl2_batch_flux_shape)."""
        v = [ctypes.c_int() for _ in range(3)]
        _bcheck(self._L.vl2_batch_flux_shape(self._h, *[ctypes.byref(x) for x in v]), self._h, lib=self._L)
        return tuple(x.value for x in v)


# ---- ABI-named module functions ----
def mesh_create(nx, mb, **kw):
    return Mesh(nx, mb, **kw)


def block_layout(mesh):
    return mesh.block_layout()


def set_prims(mesh, w, b1, b2, b3):
    return mesh.set_prims(w, b1, b2, b3)


def fill_ghosts(mesh):
    return mesh.fill_ghosts()


def step(mesh, dt):
    return mesh.step(dt)


def new_dt(mesh):
    return mesh.new_dt()


def get_cons(mesh, out=None):
    return mesh.get_cons(out)


def get_prims(mesh, out=None):
    return mesh.get_prims(out)


def divb_norm(mesh):
    return mesh.divb_norm()


def totals(mesh):
    return mesh.totals()


def batch_create(meshes):
    return Batch(meshes)
