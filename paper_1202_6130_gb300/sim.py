"""Python face of the engine: one ``Simulation`` per lattice, backed by an
``lbm_ctx`` of the CUDA library.  PyTorch supplies device memory (its caching
allocator, through the ABI's allocator callbacks) and the CUDA stream; every
step of the update runs in the library's kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib as L


class TorchAllocator:
    """lbm_allocator backed by torch's caching allocator on one device."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.live = {}
        self._alloc = L.ALLOC_FN(self._alloc_cb)
        self._free = L.FREE_FN(self._free_cb)
        self.struct = L.lbm_allocator(self._alloc, self._free, None)

    def _alloc_cb(self, nbytes, user):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        except Exception:  # out of memory -> NULL -> LBM_ENOMEM
            return None
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _free_cb(self, ptr, user):
        self.live.pop(ptr, None)


def _c64(a, shape=None):
    if a is None:
        return None
    out = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and out.shape != tuple(shape):
        out = out.reshape(shape)
    return out


class Simulation:
    """One lattice on the current CUDA device.

    Parameters mirror ``lbm_params`` (include/lbm.h); ``storage`` is one of
    "fp64", "fp32", "fp16s", "bf16s"; ``lattice`` is 9 or 21.
    """

    def __init__(self, nx: int, ny: int, lattice: int = 9, storage: str = "fp32",
                 tau: float = 1.0, G: float = -5.5, rho0: float = 1.0, psi_kind: int = 0,
                 project: bool = False, body_force=(0.0, 0.0), shift_rho: float = 0.0,
                 eos=None, check_every: int = 0, tile_rows: int = 0, stream=None,
                 use_torch_allocator: bool = True, rounding: str = "stochastic"):
        import torch
        self.lib = L.load()
        p = L.lbm_params()
        L.check(self.lib.lbm_params_default(ctypes.byref(p)))
        p.nx, p.ny, p.lattice = int(nx), int(ny), int(lattice)
        p.storage = L.STORAGE[storage] if isinstance(storage, str) else int(storage)
        p.psi_kind, p.project = int(psi_kind), int(bool(project))
        p.tau, p.G, p.rho0 = float(tau), float(G), float(rho0)
        if eos is not None:
            p.eos_theta_v, p.eos_theta_u, p.eos_theta_l, p.eos_rho1, p.eos_rho2 = map(float, eos)
        p.body_force[0], p.body_force[1] = float(body_force[0]), float(body_force[1])
        p.shift_rho = float(shift_rho)
        p.check_every, p.tile_rows = int(check_every), int(tile_rows)
        p.rounding = L.ROUNDING[rounding] if isinstance(rounding, str) else int(rounding)
        self.params = p
        self.nx, self.ny, self.Q = int(nx), int(ny), int(lattice)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.allocator = TorchAllocator(self.device) if use_torch_allocator else None
        ctx = ctypes.c_void_p()
        rc = self.lib.lbm_create(ctypes.byref(p),
                                 ctypes.byref(self.allocator.struct) if self.allocator else None,
                                 ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(ctx))
        L.check(rc, None)
        self.ctx = ctx

    # -- life cycle -----------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            self.lib.lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _chk(self, rc):
        L.check(rc, self.ctx)

    # -- state ----------------------------------------------------------------
    def set_wall(self, phi_s=None, psi_r=None, psi_a=None, G_R=0.0, G_A=0.0, epsilon=1.0,
                 u_wall=None):
        sh = (self.ny, self.nx)
        a = [_c64(phi_s, sh), _c64(psi_r, sh), _c64(psi_a, sh)]
        uw = _c64(u_wall, (2,) + sh)
        self._chk(self.lib.lbm_set_wall(self.ctx, L.dptr(a[0]), L.dptr(a[1]), L.dptr(a[2]),
                                        float(G_R), float(G_A), float(epsilon), L.dptr(uw)))

    def set_populations(self, f):
        f = _c64(f, (self.Q, self.ny, self.nx))
        self._chk(self.lib.lbm_set_populations(self.ctx, L.dptr(f)))

    def set_equilibrium(self, rho, ux=None, uy=None, dfi=None):
        sh = (self.ny, self.nx)
        rho = _c64(rho, sh)
        ux = _c64(ux if ux is not None else np.zeros(sh), sh)
        uy = _c64(uy if uy is not None else np.zeros(sh), sh)
        d = _c64(dfi, (self.Q,) + sh)
        self._chk(self.lib.lbm_set_equilibrium(self.ctx, L.dptr(rho), L.dptr(ux), L.dptr(uy),
                                               L.dptr(d)))

    def step(self, n: int = 1):
        self._chk(self.lib.lbm_step(self.ctx, int(n)))

    def sync(self):
        self._chk(self.lib.lbm_sync(self.ctx))

    # -- read-out -------------------------------------------------------------
    def moments(self, out=None):
        sh = (self.ny, self.nx)
        if out is None:
            out = (np.empty(sh), np.empty(sh), np.empty(sh))
        self._chk(self.lib.lbm_moments(self.ctx, *(L.dptr(o) for o in out)))
        return out

    def moments_device(self):
        """(rho, ux, uy) as float64 torch tensors on the device (no host sync)."""
        import torch
        t = torch.empty((3, self.ny, self.nx), dtype=torch.float64, device=self.device)
        self._chk(self.lib.lbm_moments_device(self.ctx, ctypes.c_void_p(t[0].data_ptr()),
                                              ctypes.c_void_p(t[1].data_ptr()),
                                              ctypes.c_void_p(t[2].data_ptr())))
        return t[0], t[1], t[2]

    def populations(self):
        f = np.empty((self.Q, self.ny, self.nx))
        self._chk(self.lib.lbm_get_populations(self.ctx, L.dptr(f)))
        return f

    def totals(self):
        out = np.empty(3)
        self._chk(self.lib.lbm_totals(self.ctx, L.dptr(out)))
        return out

    def steps_done(self) -> int:
        v = ctypes.c_int64()
        self._chk(self.lib.lbm_steps_done(self.ctx, ctypes.byref(v)))
        return v.value

    def clock(self):
        """(steps since the populations were set, stochastic-rounding counter,
        shift density rho_s of 16-bit storage or 0)."""
        st, rc, rs = ctypes.c_int64(), ctypes.c_uint32(), ctypes.c_double()
        self._chk(self.lib.lbm_get_clock(self.ctx, ctypes.byref(st), ctypes.byref(rc),
                                         ctypes.byref(rs)))
        return st.value, rc.value, rs.value

    def checkpoint(self) -> dict:
        """The state needed to resume bit for bit: the parameters this object
        was created with, the populations (FP64, the layout of
        set_populations) and the clock.  The wall fields are the caller's
        static inputs; set them again on the restored simulation."""
        steps, counter, rho_s = self.clock()
        p = self.params
        params = {k: getattr(p, k) for k, _ in L.lbm_params._fields_ if k != "body_force"}
        params["body_force"] = (p.body_force[0], p.body_force[1])
        return {"populations": self.populations(), "steps": steps, "rounding_counter": counter,
                "rho_s": rho_s, "params": params}

    def restore(self, ckpt: dict):
        """Sets the populations and the clock of a checkpoint.  Bit for bit
        only if this simulation has the checkpoint's parameters and, for
        16-bit storage, its shift density (``from_checkpoint`` makes one)."""
        self.set_populations(ckpt["populations"])
        self._chk(self.lib.lbm_set_clock(self.ctx, int(ckpt["steps"]),
                                         int(ckpt["rounding_counter"])))

    def save(self, path: str):
        """Writes checkpoint() to an .npz file."""
        c = self.checkpoint()
        params = c.pop("params")
        np.savez(path, **c, **{"param_" + k: np.asarray(v) for k, v in params.items()})

    @staticmethod
    def read_checkpoint(path: str) -> dict:
        with np.load(path) as z:
            c = {k: z[k] for k in z.files if not k.startswith("param_")}
            c["params"] = {k[6:]: z[k].tolist() for k in z.files if k.startswith("param_")}
        return c

    @classmethod
    def from_checkpoint(cls, ckpt, **kw):
        """A new simulation with a checkpoint's parameters (the shift density
        included), its populations and its clock.  ``ckpt``: a dict of
        checkpoint() or the path of a save() file.  Walls: call set_wall."""
        if isinstance(ckpt, str):
            ckpt = cls.read_checkpoint(ckpt)
        p = dict(ckpt["params"])
        eos = (p["eos_theta_v"], p["eos_theta_u"], p["eos_theta_l"], p["eos_rho1"], p["eos_rho2"])
        sim = cls(int(p["nx"]), int(p["ny"]), lattice=int(p["lattice"]), storage=int(p["storage"]),
                  tau=p["tau"], G=p["G"], rho0=p["rho0"], psi_kind=int(p["psi_kind"]),
                  project=bool(p["project"]), body_force=tuple(p["body_force"]),
                  shift_rho=float(ckpt["rho_s"]) if float(ckpt["rho_s"]) > 0 else p["shift_rho"],
                  eos=eos, check_every=int(p["check_every"]), tile_rows=int(p["tile_rows"]),
                  rounding=int(p["rounding"]), **kw)
        sim.restore(ckpt)
        return sim

    def layout(self) -> dict:
        lay = L.lbm_layout()
        self._chk(self.lib.lbm_get_layout(self.ctx, ctypes.byref(lay)))
        return {k: getattr(lay, k) for k, _ in L.lbm_layout._fields_}

    # -- convenience ------------------------------------------------------------
    @classmethod
    def from_workload(cls, w, storage: str = "fp32", **kw):
        """Builds, walls and initialises a simulation from an object with the
        attributes nx, ny, lattice, tau, G, rho0, body_force, rho, ux, uy, noise,
        phi_s, psi_r, psi_a, G_R, G_A, epsilon, u_wall."""
        sim = cls(w.nx, w.ny, lattice=w.lattice, storage=storage, tau=w.tau, G=w.G,
                  rho0=w.rho0, psi_kind=getattr(w, "psi_kind", 0),
                  body_force=tuple(w.body_force), **kw)
        if w.phi_s is not None or w.psi_r is not None or w.psi_a is not None:
            sim.set_wall(w.phi_s, w.psi_r, w.psi_a, w.G_R, w.G_A, w.epsilon, w.u_wall)
        sim.set_equilibrium(w.rho, w.ux, w.uy, w.noise)
        return sim


class Batch:
    """Several Simulations of one (lattice, storage) kind advanced together: one
    fused launch per chunk of up to 64 members (32 with FP64 storage) per time
    step (lbm_batch_* of
    include/lbm.h)."""

    def __init__(self, stream=None, use_torch_allocator: bool = True, device=None):
        """``stream``: the stream batch steps run on; by default a new stream, so
        that runs of steps can be captured in CUDA graphs.  Each step is ordered
        with the members' streams by the library (events both ways)."""
        import torch
        self.lib = L.load()
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        self.stream = stream if stream is not None else torch.cuda.Stream(dev)
        self.allocator = TorchAllocator(dev) if use_torch_allocator else None
        h = ctypes.c_void_p()
        L.check_batch(self.lib.lbm_batch_create(
            ctypes.byref(self.allocator.struct) if self.allocator else None,
            ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h
        self.members = []

    def _chk(self, rc):
        L.check_batch(rc, self.h)

    def add(self, sim: "Simulation"):
        self._chk(self.lib.lbm_batch_add(self.h, sim.ctx))
        self.members.append(sim)

    def remove(self, sim: "Simulation"):
        self.stream.synchronize()
        self._chk(self.lib.lbm_batch_remove(self.h, sim.ctx))
        self.members.remove(sim)

    def synchronize(self):
        self.stream.synchronize()

    def launches_per_step(self) -> int:
        """Kernel launches per batch time step (one per chunk of up to 64 members,
        32 with FP64 storage)."""
        n = ctypes.c_int32()
        self._chk(self.lib.lbm_batch_launches_per_step(self.h, ctypes.byref(n)))
        return n.value

    def set_tiling(self, tile_rows: int = 0, ctas: int = 0):
        self._chk(self.lib.lbm_batch_set_tiling(self.h, int(tile_rows), int(ctas)))

    def step(self, n: int = 1):
        self._chk(self.lib.lbm_batch_step(self.h, int(n)))

    def use_tuned(self) -> bool:
        """Adopt the tiling an earlier autotune chose for a batch of the same
        lattice, storage and size class (advances nothing); False if none."""
        found = ctypes.c_int32()
        self._chk(self.lib.lbm_batch_use_tuned(self.h, ctypes.byref(found)))
        return bool(found.value)

    def autotune(self, steps_per_trial: int = 20):
        tr, ct, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        self._chk(self.lib.lbm_batch_autotune(self.h, int(steps_per_trial), ctypes.byref(tr),
                                              ctypes.byref(ct), ctypes.byref(ms)))
        return dict(tile_rows=tr.value, ctas=ct.value, ms_per_step=ms.value)

    def close(self):
        if getattr(self, "h", None):
            self.lib.lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wall_gaussian_filter(solid: np.ndarray, lattice: int = 21, n_rep: int = 5, n_att: int = 22):
    """Appendix wall functions on the device: returns (phi_S, psi_R-bar, psi_A-bar)."""
    lib = L.load()
    solid = np.ascontiguousarray(solid, dtype=np.uint8)
    ny, nx = solid.shape
    outs = [np.empty((ny, nx)) for _ in range(3)]
    L.check(lib.lbm_wall_gaussian_filter(nx, ny, int(lattice),
                                         solid.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                         int(n_rep), int(n_att), *(L.dptr(o) for o in outs)))
    return tuple(outs)


def wall_core_tail(dist: np.ndarray, thickness, core_lambda=1.0, core_cut=4.0, tail_exp=3.0,
                   tail_cut=4.0, phi_cut=1e-16):
    """Closed-form core/tail wall fields (host helper of the library)."""
    lib = L.load()
    dist = np.ascontiguousarray(dist, dtype=np.float64)
    ny, nx = dist.shape
    th = np.ascontiguousarray(np.broadcast_to(np.asarray(thickness, dtype=np.float64).reshape(-1)
                                              if np.ndim(thickness) else thickness, (nx,)))
    outs = [np.empty((ny, nx)) for _ in range(3)]
    L.check(lib.lbm_wall_core_tail(nx, ny, L.dptr(dist), L.dptr(th), core_lambda, core_cut,
                                   tail_exp, tail_cut, phi_cut, *(L.dptr(o) for o in outs)))
    return tuple(outs)
