"""Python binding of libmhd.so (include/mhd.h): ctypes argument marshalling only.

Every step of the time step runs in the CUDA kernels of libmhd.so; this module converts arrays to
pointers and return codes to exceptions.  Host data are numpy arrays; device data are torch CUDA
tensors (their data pointers are passed with on_device = 1).  If the library is missing the import
of a Sim raises: there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OPT = {"bc_x": 1, "bc_y": 2, "bc_z": 3, "chem": 4, "precision": 5, "regul_mode": 7,
       "chem_lshield": 8, "chem_bdop": 9, "chem_xnorm": 10, "chem_taud": 11, "graph": 14,
       "heatcool": 15, "grav_g": 16, "ions": 17, "x_stage": 18}
STATUS = {0: "MHD_OK", 1: "MHD_PENDING", -1: "MHD_EINVAL", -2: "MHD_ENOMEM", -3: "MHD_ECUDA",
          -4: "MHD_ENONPHYS", -5: "MHD_ETIMEOUT", -6: "MHD_ENOTFOUND", -7: "MHD_ECAPACITY",
          -8: "MHD_ECANCELED"}
F64, F32 = 0, 1


class MHDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Fields(C.Structure):
    _fields_ = [("rho", C.c_void_p), ("mom", C.c_void_p * 3), ("E", C.c_void_p),
                ("B", C.c_void_p * 3), ("rho_h2", C.c_void_p), ("dtype", C.c_int),
                ("on_device", C.c_int)]


class Diag(C.Structure):
    _fields_ = [("sum_rho", C.c_double), ("sum_mom", C.c_double * 3), ("sum_E", C.c_double),
                ("sum_b", C.c_double * 3), ("max_div_b_h", C.c_double), ("t", C.c_double),
                ("tau_next", C.c_double), ("steps", C.c_int64), ("vel_branch", C.c_int64),
                ("error_flags", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("gamma", C.c_double),
                ("dx", C.c_double), ("precision", C.c_int), ("chem", C.c_int),
                ("bc", C.c_int * 3), ("cfl", C.c_double), ("nsteps", C.c_int), ("state", Fields)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("steps_done", C.c_int64), ("t", C.c_double),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("cells", C.c_int64)]


_lib = None


def lib():
    """Load libmhd.so (built in-tree by paper_1608_08748_gb300.build)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libmhd.so not built ({path}); run paper_1608_08748_gb300.build.build()")
        L = C.CDLL(path)
        vp, d, i = C.c_void_p, C.c_double, C.c_int
        L.mhd_create.restype = vp
        L.mhd_create.argtypes = [i, i, i, d, d]
        L.mhd_destroy.argtypes = [vp]
        L.mhd_last_error.restype = C.c_char_p
        L.mhd_set_option.argtypes = [vp, i, d]
        L.mhd_set_stream.argtypes = [vp, vp]
        L.mhd_set_state.argtypes = [vp, C.POINTER(Fields)]
        L.mhd_set_face_B.argtypes = [vp, vp, vp, vp, i]
        L.mhd_get_state.argtypes = [vp, C.POINTER(Fields)]
        L.mhd_get_full.argtypes = [vp, vp, vp, vp, vp, i]
        L.mhd_set_full.argtypes = [vp, vp, vp, vp, vp, i]
        L.mhd_step.argtypes = [vp, d, C.POINTER(d)]
        L.mhd_advance.argtypes = [vp, d, d, i, C.POINTER(i)]
        L.mhd_sync.argtypes = [vp]
        L.mhd_stage.argtypes = [vp, i, d]
        L.mhd_diagnostics.argtypes = [vp, C.POINTER(Diag)]
        L.mhd_bytes_needed.restype = C.c_size_t
        L.mhd_bytes_needed.argtypes = [i, i, i, i, i]
        L.mhd_profile.argtypes = [vp, d, i, C.POINTER(d), C.POINTER(C.c_int64)]
        L.mhd_launches_per_step.argtypes = [vp]
        L.mhd_get_potential.argtypes = [vp, vp]
        L.mhd_set_ions.argtypes = [vp, vp, i]
        L.mhd_probe_fma_peak.argtypes = [i, i, C.POINTER(d)]
        L.mhd_get_ions.argtypes = [vp, vp, i]
        L.mhd_batch_create.restype = vp
        L.mhd_batch_create.argtypes = [C.POINTER(vp), i]
        L.mhd_batch_destroy.argtypes = [vp]
        L.mhd_batch_step.argtypes = [vp, d]
        L.mhd_batch_sync.argtypes = [vp]
        L.mhd_batch_tune.argtypes = [vp, d, i, C.POINTER(d)]
        L.mhd_batch_get_shape.argtypes = [vp, i, C.POINTER(i), C.POINTER(i)]
        L.mhd_batch_set_shape.argtypes = [vp, i, i, i]
        L.mhd_batch_profile.argtypes = [vp, d, i, C.POINTER(d), C.POINTER(C.c_int64)]
        L.mhd_server_create.restype = vp
        L.mhd_server_create.argtypes = [C.c_size_t, i]
        L.mhd_server_destroy.argtypes = [vp]
        L.mhd_submit.restype = C.c_int64
        L.mhd_submit.argtypes = [vp, C.POINTER(Request)]
        L.mhd_poll.argtypes = [vp, C.c_int64, C.POINTER(Result)]
        L.mhd_fetch.argtypes = [vp, C.c_int64, C.POINTER(Fields)]
        L.mhd_server_drain.argtypes = [vp, d]
        L.mhd_server_clock.restype = d
        L.mhd_server_clock.argtypes = [vp]
        L.mhd_server_stats.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(i)]
        L.mhd_server_set_policy.argtypes = [vp, i]
        L.mhd_cancel.argtypes = [vp, C.c_int64]
        L.mhd_server_pause.argtypes = [vp, i]
        L.mhd_server_set_budget.argtypes = [vp, C.c_size_t]
        L.mhd_server_set_bulk_cells.argtypes = [vp, C.c_int64]
        L.mhd_batch_query.argtypes = [vp]
        L.mhd_batch_set_priority.argtypes = [vp, i]
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise MHDError(rc, lib().mhd_last_error().decode())


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """(pointer, on_device, keepalive) of a numpy array or torch tensor of the given dtype."""
    if _is_torch(x):
        import torch
        want = torch.float64 if dtype == F64 else torch.float32
        if x.dtype != want or not x.is_contiguous():
            raise ValueError("device tensors must be contiguous and of the requested dtype")
        return x.data_ptr(), int(x.is_cuda), x
    want = np.float64 if dtype == F64 else np.float32
    a = np.ascontiguousarray(x, dtype=want)
    return a.ctypes.data, 0, a


class Sim:
    """One simulation box on the current CUDA device (all memory owned by libmhd.so)."""

    def __init__(self, nx, ny, nz, gamma, dx, **options):
        self.L = lib()
        self.shape = (nz, ny, nx)
        self.h = self.L.mhd_create(nx, ny, nz, float(gamma), float(dx))
        if not self.h:
            raise MHDError(-1, self.L.mhd_last_error().decode())
        for k, v in options.items():
            self.set_option(k, v)

    def close(self):
        if getattr(self, "h", None):
            self.L.mhd_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def set_option(self, key, value):
        _check(self.L.mhd_set_option(self.h, OPT[key], float(value)))

    def set_stream(self, stream_ptr):
        _check(self.L.mhd_set_stream(self.h, stream_ptr))

    def _fields(self, rho, mom, E, B, rho_h2, dtype):
        keep = []
        f = Fields()
        vals = []
        on_dev = set()
        for x in [rho, mom[0], mom[1], mom[2], E, B[0], B[1], B[2], rho_h2]:
            if x is None:
                vals.append(None)
                continue
            p, dev, k = _ptr(x, dtype)
            keep.append(k)
            on_dev.add(dev)
            vals.append(p)
        if len(on_dev) > 1:
            raise ValueError("all fields must be on the host or all on the device")
        f.rho = vals[0]
        for q in range(3):
            f.mom[q] = vals[1 + q]
            f.B[q] = vals[5 + q]
        f.E = vals[4]
        f.rho_h2 = vals[8]
        f.dtype = dtype
        f.on_device = on_dev.pop() if on_dev else 0
        return f, keep

    def set_state(self, rho, mom, E, B, rho_h2=None, dtype=None):
        if dtype is None:
            dtype = F32 if getattr(rho, "dtype", None) in (np.float32,) or str(getattr(rho, "dtype", "")) == "torch.float32" else F64
        f, keep = self._fields(rho, mom, E, B, rho_h2, dtype)
        _check(self.L.mhd_set_state(self.h, C.byref(f)))

    def set_face_B(self, bx, by, bz):
        ptrs = [_ptr(x, F64) for x in (bx, by, bz)]
        _check(self.L.mhd_set_face_B(self.h, ptrs[0][0], ptrs[1][0], ptrs[2][0], ptrs[0][1]))

    def get_state(self, dtype=F64, out=None):
        """Copy the state out: numpy arrays by default, or into `out` (dict of arrays/tensors)."""
        npdt = np.float64 if dtype == F64 else np.float32
        if out is None:
            out = {"rho": np.empty(self.shape, npdt), "mom": np.empty((3,) + self.shape, npdt),
                   "E": np.empty(self.shape, npdt), "B": np.empty((3,) + self.shape, npdt),
                   "rho_h2": np.empty(self.shape, npdt)}
        f, keep = self._fields(out["rho"], out["mom"], out["E"], out["B"], out.get("rho_h2"), dtype)
        _check(self.L.mhd_get_state(self.h, C.byref(f)))
        return out

    def get_full(self):
        out = [np.empty(self.shape) for _ in range(4)]
        _check(self.L.mhd_get_full(self.h, *[o.ctypes.data for o in out], 0))
        return {"eint": out[0], "bface": np.stack(out[1:])}

    def set_full(self, eint, bface):
        a = [np.ascontiguousarray(x, dtype=np.float64) for x in (eint, bface[0], bface[1], bface[2])]
        _check(self.L.mhd_set_full(self.h, *[x.ctypes.data for x in a], 0))

    def step(self, cfl, sync=True):
        if sync:
            dt = C.c_double(0.0)
            _check(self.L.mhd_step(self.h, float(cfl), C.byref(dt)))
            return dt.value
        _check(self.L.mhd_step(self.h, float(cfl), None))
        return None

    def advance(self, cfl, t_end, max_steps=1 << 30):
        n = C.c_int(0)
        _check(self.L.mhd_advance(self.h, float(cfl), float(t_end), int(max_steps), C.byref(n)))
        return n.value

    def sync(self):
        _check(self.L.mhd_sync(self.h))

    def stage(self, which, tau):
        _check(self.L.mhd_stage(self.h, int(which), float(tau)))

    def set_ions(self, rho_hp):
        """rho_H+ of every cell (float64; numpy or a CUDA tensor); after set_state, which zeroes it."""
        p, on_dev, keep = _ptr(rho_hp, F64)
        _check(self.L.mhd_set_ions(self.h, p, on_dev))
        del keep

    def get_ions(self):
        out = np.empty(self.shape)
        _check(self.L.mhd_get_ions(self.h, out.ctypes.data, 0))
        return out

    def potential(self):
        """Sec. 2.10 gravitational potential of the current density (needs the grav_g option)."""
        out = np.empty(self.shape)
        _check(self.L.mhd_get_potential(self.h, out.ctypes.data))
        return out

    def diagnostics(self):
        d = Diag()
        _check(self.L.mhd_diagnostics(self.h, C.byref(d)))
        return {"rho": d.sum_rho, "mx": d.sum_mom[0], "my": d.sum_mom[1], "mz": d.sum_mom[2],
                "E": d.sum_E, "bx": d.sum_b[0], "by": d.sum_b[1], "bz": d.sum_b[2],
                "max_div_b_h": d.max_div_b_h, "t": d.t, "tau_next": d.tau_next, "steps": d.steps,
                "vel_branch": d.vel_branch, "error_flags": d.error_flags}


def bytes_needed(nx, ny, nz, precision=0, chem=1):
    return lib().mhd_bytes_needed(nx, ny, nz, precision, chem)


def probe_fma_peak(fp64=True, iters=None):
    """Measured FMA peak of the current GPU in TFLOP/s (mhd_probe_fma_peak), FP64 or FP32."""
    if iters is None:
        iters = 20000 if fp64 else 400000
    out = C.c_double(0.0)
    _check(lib().mhd_probe_fma_peak(int(bool(fp64)), int(iters), C.byref(out)))
    return out.value


def log_steps(sim, cfl, steps, path):
    """Advance `sim` by `steps` steps, appending one JSON line per step to `path`: the step number,
    t, tau, the FP64 sums (rho, m, rho E, b), max |div b| h, the cumulative velocity-branch count of
    the regularisation and the error flags (mhd_diagnostics after each step, which synchronises)."""
    import json
    with open(path, "a") as f:
        for _ in range(steps):
            tau = sim.step(cfl)
            d = sim.diagnostics()
            rec = {"step": int(d["steps"]), "t": d["t"], "tau": tau}
            rec.update({k: d[k] for k in ["rho", "mx", "my", "mz", "E", "bx", "by", "bz", "max_div_b_h"]})
            rec.update(vel_branch=int(d["vel_branch"]), error_flags=int(d["error_flags"]))
            f.write(json.dumps(rec) + "\n")


def from_ic(ic, **options):
    """Sim loaded from an initial-condition dict of paper_1608_08748_gb300.inputs."""
    nz, ny, nx = ic["rho"].shape
    opts = dict(ic.get("options", {}))
    opts.update(options)
    s = Sim(nx, ny, nz, ic["gamma"], ic["dx"], **opts)
    s.set_state(ic["rho"], ic["mom"], ic["E"], ic["B"], ic.get("rho_h2"))
    if ic.get("rho_hp") is not None:
        s.set_ions(ic["rho_hp"])
    if "bface" in ic:
        s.set_face_B(*ic["bface"])
    return s


KERNEL_CLASSES = ["prim", "euler_face", "edges", "euler_update", "lag_face", "lag_update", "post",
                  "small"]


def _profile_dict(ms, n):
    return {k: {"ms_total": ms[c], "launches": int(n[c])} for c, k in enumerate(KERNEL_CLASSES)}


def profile(sim, cfl, steps):
    """Per kernel class CUDA-event time of `steps` launched steps of one sim (advances it)."""
    ms = (C.c_double * 8)()
    n = (C.c_int64 * 8)()
    _check(sim.L.mhd_profile(sim.h, float(cfl), int(steps), ms, n))
    return _profile_dict(ms, n)


class Batch:
    """Sims advanced together, one launch per kernel class over all their boxes."""

    def __init__(self, sims):
        self.L = lib()
        self.sims = list(sims)  # keep the members alive
        arr = (C.c_void_p * len(self.sims))(*[x.h for x in self.sims])
        self.h = self.L.mhd_batch_create(arr, len(self.sims))
        if not self.h:
            raise MHDError(-1, self.L.mhd_last_error().decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.mhd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def step(self, cfl):
        _check(self.L.mhd_batch_step(self.h, float(cfl)))

    def sync(self):
        _check(self.L.mhd_batch_sync(self.h))

    def tune(self, cfl, reps=2):
        best = C.c_double(0.0)
        _check(self.L.mhd_batch_tune(self.h, float(cfl), int(reps), C.byref(best)))
        return best.value

    def shape(self, kernel_class):
        b, g = C.c_int(0), C.c_int(0)
        _check(self.L.mhd_batch_get_shape(self.h, KERNEL_CLASSES.index(kernel_class), C.byref(b), C.byref(g)))
        return b.value, g.value

    def set_shape(self, kernel_class, block, grid_mult):
        _check(self.L.mhd_batch_set_shape(self.h, KERNEL_CLASSES.index(kernel_class), int(block), int(grid_mult)))

    def profile(self, cfl, steps):
        ms = (C.c_double * 8)()
        n = (C.c_int64 * 8)()
        _check(self.L.mhd_batch_profile(self.h, float(cfl), int(steps), ms, n))
        return _profile_dict(ms, n)


class Server:
    """Continuous-batching request server of libmhd.so (scheduler thread in the library)."""

    def __init__(self, hbm_budget_bytes, max_active=64):
        self.L = lib()
        self.h = self.L.mhd_server_create(int(hbm_budget_bytes), int(max_active))
        if not self.h:
            raise MHDError(-1, self.L.mhd_last_error().decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.mhd_server_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def set_policy(self, policy):
        """Admission order: "fifo" (the default) or "smallest_work" (fewest cells x steps first)."""
        _check(self.L.mhd_server_set_policy(self.h, {"fifo": 0, "smallest_work": 1}[policy]))

    def cancel(self, rid):
        """Cancel a waiting or running request (its status becomes MHD_ECANCELED)."""
        _check(self.L.mhd_cancel(self.h, int(rid)))

    def pause(self, paused=True):
        """Hold (True) or resume (False) the admission of waiting requests."""
        _check(self.L.mhd_server_pause(self.h, int(bool(paused))))

    def set_budget(self, hbm_budget_bytes):
        """New HBM budget; waiting requests that can no longer fit fail with MHD_ECAPACITY."""
        _check(self.L.mhd_server_set_budget(self.h, int(hbm_budget_bytes)))

    def set_bulk_cells(self, cells):
        """Requests of at least `cells` cells run in the low-priority bulk lane."""
        _check(self.L.mhd_server_set_bulk_cells(self.h, int(cells)))

    def drain_rc(self, timeout_s):
        """mhd_server_drain's status (MHD_OK or MHD_ETIMEOUT) without raising."""
        return self.L.mhd_server_drain(self.h, float(timeout_s))

    def submit(self, ic, nsteps, cfl=0.4, precision=1):
        """Queue a request built from an initial-condition dict; returns its id."""
        nz, ny, nx = ic["rho"].shape
        opts = ic.get("options", {})
        r = Request()
        r.nx, r.ny, r.nz = nx, ny, nz
        r.gamma, r.dx = float(ic["gamma"]), float(ic["dx"])
        r.precision, r.chem = int(precision), int(opts.get("chem", 0))
        r.bc[0], r.bc[1], r.bc[2] = int(opts.get("bc_x", 0)), int(opts.get("bc_y", 0)), int(opts.get("bc_z", 0))
        r.cfl, r.nsteps = float(cfl), int(nsteps)
        keep = []
        f = Fields()
        vals = []
        for x in [ic["rho"], ic["mom"][0], ic["mom"][1], ic["mom"][2], ic["E"], ic["B"][0], ic["B"][1],
                  ic["B"][2], ic.get("rho_h2")]:
            if x is None:
                vals.append(None)
                continue
            a = np.ascontiguousarray(x, dtype=np.float64)
            keep.append(a)
            vals.append(a.ctypes.data)
        f.rho, f.E, f.rho_h2 = vals[0], vals[4], vals[8]
        for q in range(3):
            f.mom[q], f.B[q] = vals[1 + q], vals[5 + q]
        f.dtype, f.on_device = F64, 0
        r.state = f
        rid = self.L.mhd_submit(self.h, C.byref(r))
        if rid < 0:
            raise MHDError(int(rid), self.L.mhd_last_error().decode())
        return rid

    def poll(self, rid):
        res = Result()
        rc = self.L.mhd_poll(self.h, int(rid), C.byref(res))
        out = {k: getattr(res, k) for k, _ in Result._fields_}
        return rc, out

    def fetch(self, rid, shape):
        out = {"rho": np.empty(shape), "mom": np.empty((3,) + tuple(shape)), "E": np.empty(shape),
               "B": np.empty((3,) + tuple(shape)), "rho_h2": np.empty(shape)}
        f = Fields()
        f.rho, f.E, f.rho_h2 = out["rho"].ctypes.data, out["E"].ctypes.data, out["rho_h2"].ctypes.data
        for q in range(3):
            f.mom[q] = out["mom"][q].ctypes.data
            f.B[q] = out["B"][q].ctypes.data
        f.dtype, f.on_device = F64, 0
        _check(self.L.mhd_fetch(self.h, int(rid), C.byref(f)))
        return out

    def drain(self, timeout_s=600.0):
        _check(self.L.mhd_server_drain(self.h, float(timeout_s)))

    def clock(self):
        return self.L.mhd_server_clock(self.h)

    def stats(self):
        it, pb, pa = C.c_int64(0), C.c_int64(0), C.c_int(0)
        _check(self.L.mhd_server_stats(self.h, C.byref(it), C.byref(pb), C.byref(pa)))
        return {"iterations": it.value, "peak_bytes": pb.value, "peak_active": pa.value}
