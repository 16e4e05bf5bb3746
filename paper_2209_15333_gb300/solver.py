"""Python handle around one ``cfd_ctx`` (include/cfd.h).

Host arrays are numpy float64; device arrays are torch CUDA tensors (used only
for device memory and streams).  All arithmetic happens in the CUDA library.
"""
import ctypes as C

import numpy as np

from . import _lib as L


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a):
    """(pointer, on_device) for a numpy array or a torch tensor."""
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr()), int(a.is_cuda)
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return C.c_void_p(a.ctypes.data), 0


def to_bf16_bits(a):
    """float32 -> bf16 bit patterns (uint16), round to nearest even."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
    return np.ascontiguousarray(r)


def from_bf16_bits(b):
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


class Solver:
    def __init__(self, shape, metrics, *, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), stream=None, **params):
        """shape = (nx, ny, nz); metrics: numpy/torch (10,), (10, ny, nx) or (10, nz, ny, nx)."""
        nx, ny, nz = shape
        self.shape = (nz, ny, nx)
        m = metrics
        ndim = m.dim() if _is_torch(m) else np.asarray(m).ndim
        layout = {1: L.METRICS_UNIFORM, 3: L.METRICS_2D, 4: L.METRICS_3D}[ndim]
        if not _is_torch(m):
            m = np.ascontiguousarray(m, dtype=np.float64)
        self._metrics = m
        self.grid = L.make_grid(nx, ny, nz, bc_lo, bc_hi, layout)
        self.params = L.default_params(**params)
        self.ctx = C.c_void_p()
        mp, mdev = _ptr(m)
        if stream is None:
            stream_ptr = None
        else:
            stream_ptr = C.c_void_p(getattr(stream, "cuda_stream", stream))
        L.check(L.lib().cfd_create(C.byref(self.ctx), C.byref(self.grid), mp, mdev, C.byref(self.params),
                                   stream_ptr))

    # ---- state ----
    def set_state(self, U, block=0):
        p, dev = _ptr(U)
        L.check(L.lib().cfd_set_state(self.ctx, block, p, dev), self.ctx)

    def get_state(self, out=None, block=0):
        if out is None:
            out = np.empty((5,) + self.shape)
        p, dev = _ptr(out)
        L.check(L.lib().cfd_get_state(self.ctx, block, p, dev), self.ctx)
        return out

    def rhs(self, out=None, block=0):
        if out is None:
            out = np.empty((5,) + self.shape)
        p, dev = _ptr(out)
        L.check(L.lib().cfd_rhs(self.ctx, block, p, dev), self.ctx)
        return out

    def step(self, dt, nsteps=1):
        L.check(L.lib().cfd_step(self.ctx, dt, nsteps), self.ctx)

    def cfl_dt(self, cfl=0.5, block=0):
        dt = C.c_double()
        L.check(L.lib().cfd_cfl_dt(self.ctx, block, cfl, C.byref(dt)), self.ctx)
        return dt.value

    def flags(self, block=0):
        out = np.empty(self.shape, dtype=np.uint8)
        L.check(L.lib().cfd_get_flags(self.ctx, block, C.c_void_p(out.ctypes.data), 0), self.ctx)
        return out

    def force_flags(self, cls, block=0):
        if cls is None:
            L.check(L.lib().cfd_force_flags(self.ctx, block, None, 0), self.ctx)
            return
        c = np.ascontiguousarray(cls, dtype=np.uint8)
        self._forced = c
        L.check(L.lib().cfd_force_flags(self.ctx, block, C.c_void_p(c.ctypes.data), 0), self.ctx)

    def set_inflow(self, prim):
        p = np.ascontiguousarray(prim, dtype=np.float64)
        L.check(L.lib().cfd_set_inflow(self.ctx, C.c_void_p(p.ctypes.data)), self.ctx)

    def set_blowing(self, amp, x0, x1, omega, m, Lz, wall_x, wall_z):
        wx = np.ascontiguousarray(wall_x, dtype=np.float64)
        wz = np.ascontiguousarray(wall_z, dtype=np.float64)
        L.check(L.lib().cfd_set_blowing(self.ctx, amp, x0, x1, omega, m, Lz, C.c_void_p(wx.ctypes.data),
                                        C.c_void_p(wz.ctypes.data)), self.ctx)

    def time(self):
        t = C.c_double()
        L.check(L.lib().cfd_get_time(self.ctx, C.byref(t)), self.ctx)
        return t.value

    def set_time(self, t):
        L.check(L.lib().cfd_set_time(self.ctx, t), self.ctx)

    def sync(self, timeout_s=60.0):
        L.check(L.lib().cfd_sync(self.ctx, timeout_s), self.ctx)

    def profile_stage(self, reps=3):
        """Mean ms per right-hand-side evaluation of each kernel (events)."""
        ms = (C.c_double * 6)()
        L.check(L.lib().cfd_profile_stage(self.ctx, reps, ms), self.ctx)
        names = ["prim", "sensor", "visc_flux", "sweep_xi", "sweep_eta", "sweep_zeta"]
        return dict(zip(names, list(ms)))

    def set_sweep_variant(self, dir, kind, param):
        L.check(L.lib().cfd_set_sweep_variant(self.ctx, dir, kind, param), self.ctx)

    def sweep_variant(self, dir):
        k, p = C.c_int(), C.c_int()
        L.check(L.lib().cfd_get_sweep_variant(self.ctx, dir, C.byref(k), C.byref(p)), self.ctx)
        return k.value, p.value

    def set_sensor_mlp(self, w1, w2, w3, b1, b2, b3, conf_min=0.0):
        """Learned sensor weights (any float arrays; rounded to bf16 here):
        w1 [32,42], w2 [32,32], w3 [3,32], biases [32], [32], [3]."""
        if w1 is None:
            L.check(L.lib().cfd_set_sensor_mlp(self.ctx, None, None, 0.0), self.ctx)
            return
        w = np.concatenate([np.asarray(a, np.float32).ravel() for a in (w1, w2, w3)])
        self._mlp_w = to_bf16_bits(w)
        self._mlp_b = np.concatenate([np.asarray(a, np.float32).ravel() for a in (b1, b2, b3)]).astype(np.float32)
        L.check(L.lib().cfd_set_sensor_mlp(self.ctx, C.c_void_p(self._mlp_w.ctypes.data),
                                           C.c_void_p(self._mlp_b.ctypes.data), float(conf_min)), self.ctx)

    def sensor_features(self, block=0):
        shp = self.shapes[block] if hasattr(self, "shapes") else self.shape
        out = np.empty((42,) + shp, dtype=np.float32)
        L.check(L.lib().cfd_sensor_features(self.ctx, block, C.c_void_p(out.ctypes.data), 0), self.ctx)
        return out

    def sensor_fallbacks(self):
        c = C.c_ulonglong()
        L.check(L.lib().cfd_sensor_fallbacks(self.ctx, C.byref(c)), self.ctx)
        return c.value

    def launches(self):
        return L.lib().cfd_launch_count(self.ctx)

    def close(self):
        if self.ctx:
            L.lib().cfd_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class BatchSolver(Solver):
    """Ensemble of independent blocks of uneven sizes (cfd_create_batch).

    shapes: list of (nx, ny, nz); metrics: list of metric arrays; params: list
    of keyword dicts (one per block); bcs: optional list of (bc_lo, bc_hi).
    """

    def __init__(self, shapes, metrics, params, *, bcs=None, stream=None):
        nb = len(shapes)
        self.shapes = [(nz, ny, nx) for (nx, ny, nz) in shapes]
        self.shape = self.shapes[0]
        grids = (L.CfdGrid * nb)()
        prms = (L.CfdParams * nb)()
        self._metrics = []
        mptrs = (C.c_void_p * nb)()
        dev_flags = set()
        for b in range(nb):
            nx, ny, nz = shapes[b]
            m = metrics[b]
            ndim = m.dim() if _is_torch(m) else np.asarray(m).ndim
            layout = {1: L.METRICS_UNIFORM, 3: L.METRICS_2D, 4: L.METRICS_3D}[ndim]
            if not _is_torch(m):
                m = np.ascontiguousarray(m, dtype=np.float64)
            self._metrics.append(m)
            lo, hi = bcs[b] if bcs else ((0, 0, 0), (0, 0, 0))
            grids[b] = L.make_grid(nx, ny, nz, lo, hi, layout)
            prms[b] = L.default_params(**params[b])
            p, dev = _ptr(m)
            mptrs[b] = p
            dev_flags.add(dev)
        if len(dev_flags) != 1:
            raise ValueError("metrics must be all on the host or all on the device")
        self.ctx = C.c_void_p()
        stream_ptr = None if stream is None else C.c_void_p(getattr(stream, "cuda_stream", stream))
        L.check(L.lib().cfd_create_batch(C.byref(self.ctx), nb, grids, mptrs, dev_flags.pop(), prms, stream_ptr))
        self.nblocks = nb

    def get_state(self, out=None, block=0):
        if out is None:
            out = np.empty((5,) + self.shapes[block])
        return super().get_state(out, block)

    def set_halo_links(self, links):
        """links: int array [nblocks][3][2] (neighbour across face (d, side),
        -1 for none), or None; see cfd_set_halo_links."""
        if links is None:
            L.check(L.lib().cfd_set_halo_links(self.ctx, None), self.ctx)
            return
        a = np.ascontiguousarray(links, dtype=np.int32)
        assert a.shape == (len(self.shapes), 3, 2)
        L.check(L.lib().cfd_set_halo_links(self.ctx, C.c_void_p(a.ctypes.data)), self.ctx)

    def rhs(self, out=None, block=0):
        if out is None:
            out = np.empty((5,) + self.shapes[block])
        return super().rhs(out, block)

    def flags(self, block=0):
        out = np.empty(self.shapes[block], dtype=np.uint8)
        L.check(L.lib().cfd_get_flags(self.ctx, block, C.c_void_p(out.ctypes.data), 0), self.ctx)
        return out

    def batch_variants(self):
        """The kernel variants the ensemble runs, as (kind, param) per
        direction: viscous fluxes, xi, eta, zeta (cfd_get_sweep_variant)."""
        return {name: self.sweep_variant(d) for name, d in (("visc", 0), ("xi", 3), ("eta", 1), ("zeta", 2))}
