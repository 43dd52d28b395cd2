"""ctypes wrapper of the FP64 CPU oracle (``mhd_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this module; the CUDA library never does.  It compiles ``mhd_oracle.c`` with gcc
(-O2 -ffp-contract=off -fopenmp) into ``oracle/_build/`` on first use.

The oracle follows the paper (arXiv:1608.08748) section by section; see the header of
``mhd_oracle.c`` for the equations it implements and the readings it takes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OPT = {
    "bc_x": 1, "bc_y": 2, "bc_z": 3, "chem": 4, "step4_as_written": 5, "iface_edge": 6,
    "regul_mode": 7, "chem_lshield": 8, "chem_bdop": 9, "chem_xnorm": 10, "chem_taud": 11,
    "threads": 12, "heatcool": 13, "grav_g": 14, "ions": 15,
}
OK, EINVAL, ENOMEM, ENONPHYS = 0, -1, -2, -4

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent); returns its path."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            os.makedirs(_BUILD, exist_ok=True)
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                   "-shared", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        vp, d, i = C.c_void_p, C.c_double, C.c_int
        L.osim_create.restype = vp
        L.osim_create.argtypes = [i, i, i, d, d]
        L.osim_destroy.argtypes = [vp]
        L.osim_set_option.argtypes = [vp, i, d]
        L.osim_set_state.argtypes = [vp] + [_dp] * 8 + [C.c_void_p]
        L.osim_set_face_B.argtypes = [vp, _dp, _dp, _dp]
        L.osim_get_state.argtypes = [vp] + [_dp] * 8 + [C.c_void_p]
        L.osim_get_full.argtypes = [vp, _dp, _dp, _dp, _dp]
        L.osim_set_full.argtypes = [vp, _dp, _dp, _dp, _dp]
        L.osim_tau.restype = d
        L.osim_tau.argtypes = [vp, d]
        L.osim_step.argtypes = [vp, d, d, C.POINTER(d)]
        L.osim_advance.argtypes = [vp, d, d, i, C.POINTER(i)]
        L.osim_stage.argtypes = [vp, i, d]
        L.osim_time.restype = d
        L.osim_time.argtypes = [vp]
        L.osim_nsteps.restype = C.c_long
        L.osim_nsteps.argtypes = [vp]
        L.osim_diag.argtypes = [vp, _dp]
        L.o_ppm.argtypes = [_dp, i, _dp]
        L.o_step4.argtypes = [_dp, _dp]
        L.o_avg.restype = d
        L.o_avg.argtypes = [_dp, d, i]
        L.o_eigen.argtypes = [_dp, _dp, _dp, _dp, _dp]
        L.o_face_solve.argtypes = [_dp, _dp, d, _dp, _dp, d, i, i, _dp]
        L.o_cfl_denominator.restype = d
        L.o_cfl_denominator.argtypes = [_dp]
        L.o_gamma_eff.restype = d
        L.o_gamma_eff.argtypes = [d, d]
        L.osim_chem_cell.argtypes = [vp, d, d, d, d, _dp]
        L.osim_heatcool_cell.argtypes = [vp, d, d, d, d, _dp]
        L.osim_potential.argtypes = [vp, _dp]
        L.osim_chem_rates.argtypes = [vp, d, d, d, _dp]
        L.osim_set_ions.argtypes = [vp, _dp]
        L.osim_get_ions.argtypes = [vp, _dp]
        L.osim_chem_cell_ions.argtypes = [vp, d, d, d, d, d, _dp]
        L.osim_heatcool_cell_ions.argtypes = [vp, d, d, d, d, d, _dp]
        L.o_ion_rates.argtypes = [d, d, d, d, _dp]
        L.o_gamma_eff_ions.restype = d
        L.o_gamma_eff_ions.argtypes = [d, d, d]
        L.o_temperature.restype = d
        L.o_temperature.argtypes = [d, d, d, d]
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Sim:
    """One oracle simulation box: fields are (nz, ny, nx) C-order float64 arrays."""

    def __init__(self, nx, ny, nz, gamma, dx, **options):
        self.L = lib()
        self.shape = (nz, ny, nx)
        self.h = self.L.osim_create(nx, ny, nz, float(gamma), float(dx))
        if not self.h:
            raise ValueError("osim_create rejected its arguments")
        for k, v in options.items():
            self.set_option(k, v)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.osim_destroy(h)
            self.h = None

    def set_option(self, key, value):
        rc = self.L.osim_set_option(self.h, OPT[key], float(value))
        if rc != OK:
            raise ValueError(f"option {key}={value} rejected ({rc})")

    def set_state(self, rho, mom, E, B, rho_h2=None):
        a = [_f64(x).reshape(self.shape) for x in (rho, mom[0], mom[1], mom[2], E, B[0], B[1], B[2])]
        h2 = _f64(rho_h2).reshape(self.shape) if rho_h2 is not None else None
        rc = self.L.osim_set_state(self.h, *a, h2.ctypes.data if h2 is not None else None)
        if rc != OK:
            raise RuntimeError(f"set_state failed ({rc})")

    def set_face_B(self, bx, by, bz):
        a = [_f64(x).reshape(self.shape) for x in (bx, by, bz)]
        self.L.osim_set_face_B(self.h, *a)

    def get_state(self):
        out = [np.empty(self.shape) for _ in range(9)]
        self.L.osim_get_state(self.h, *out[:8], out[8].ctypes.data)
        rho, mx, my, mz, E, Bx, By, Bz, h2 = out
        return {"rho": rho, "mom": np.stack([mx, my, mz]), "E": E, "B": np.stack([Bx, By, Bz]),
                "rho_h2": h2}

    def get_full(self):
        out = [np.empty(self.shape) for _ in range(4)]
        self.L.osim_get_full(self.h, *out)
        return {"eint": out[0], "bface": np.stack(out[1:])}

    def set_full(self, eint, bface):
        a = [_f64(x).reshape(self.shape) for x in (eint, bface[0], bface[1], bface[2])]
        self.L.osim_set_full(self.h, *a)

    def tau(self, cfl):
        return self.L.osim_tau(self.h, float(cfl))

    def step(self, cfl, t_end=0.0):
        dt = C.c_double(0.0)
        rc = self.L.osim_step(self.h, float(cfl), float(t_end), C.byref(dt))
        if rc != OK:
            raise RuntimeError(f"oracle step failed ({rc})")
        return dt.value

    def stage(self, which, tau):
        rc = self.L.osim_stage(self.h, int(which), float(tau))
        if rc != OK:
            raise RuntimeError(f"oracle stage {which} failed ({rc})")

    def advance(self, cfl, t_end, max_steps=1 << 30):
        n = C.c_int(0)
        rc = self.L.osim_advance(self.h, float(cfl), float(t_end), int(max_steps), C.byref(n))
        if rc != OK:
            raise RuntimeError(f"oracle advance failed ({rc})")
        return n.value

    @property
    def t(self):
        return self.L.osim_time(self.h)

    @property
    def nsteps(self):
        return self.L.osim_nsteps(self.h)

    def diag(self):
        out = np.zeros(10)
        self.L.osim_diag(self.h, out)
        keys = ["rho", "mx", "my", "mz", "E", "bx", "by", "bz", "max_div_b_h", "vel_branch"]
        return dict(zip(keys, out))

    def chem_cell(self, rho, eint, rh2, tau):
        out = np.zeros(8)
        self.L.osim_chem_cell(self.h, float(rho), float(eint), float(rh2), float(tau), out)
        return dict(zip(["rho_h2", "T", "k1p", "k2", "k3", "k4", "C", "D"], out))

    def potential(self):
        """Sec. 2.10 potential of the current density (needs the grav_g option)."""
        out = np.zeros(self.shape)
        if self.L.osim_potential(self.h, out.reshape(-1)) != OK:
            raise ValueError("no self-gravity (grav_g = 0)")
        return out

    def heatcool_cell(self, rho, eint, rh2, tau):
        """Sec. 2.8 heating/cooling of one cell: the change of rho E and rho eps (code units) and the
        terms in erg cm^-3 s^-1."""
        out = np.zeros(7)
        self.L.osim_heatcool_cell(self.h, float(rho), float(eint), float(rh2), float(tau), out)
        return dict(zip(["delta", "T", "G1", "L2", "L3", "G4", "net"], out))

    def chem_rates(self, T, nH, nH2):
        out = np.zeros(7)
        self.L.osim_chem_rates(self.h, float(T), float(nH), float(nH2), out)
        return dict(zip(["k1p", "k2", "k3", "k4", "C", "D", "T"], out))

    def set_ions(self, rho_hp):
        """rho_H+ (= n_H+, code density units) of every cell; call after set_state."""
        self.L.osim_set_ions(self.h, _f64(rho_hp).reshape(-1))

    def get_ions(self):
        out = np.zeros(self.shape)
        self.L.osim_get_ions(self.h, out.reshape(-1))
        return out

    def chem_cell_ions(self, rho, eint, rh2, rhp, tau):
        """Sec. 2.7 chemistry of one cell with H+ (reactions 5-8 when the ions option is on)."""
        out = np.zeros(15)
        self.L.osim_chem_cell_ions(self.h, float(rho), float(eint), float(rh2), float(rhp), float(tau), out)
        keys = ["rho_h2", "rho_hp", "T", "k1p", "k2", "k3", "k4", "C", "D", "k5", "k6", "k7", "k8",
                "C_hp", "D_hp"]
        return dict(zip(keys, out))

    def heatcool_cell_ions(self, rho, eint, rh2, rhp, tau):
        out = np.zeros(11)
        self.L.osim_heatcool_cell_ions(self.h, float(rho), float(eint), float(rh2), float(rhp), float(tau), out)
        keys = ["delta", "T", "G1", "L2", "L3", "G4", "G5", "L6", "L7", "L8", "net"]
        return dict(zip(keys, out))


def ppm(q5, step4_as_written=False):
    out = np.zeros(4)
    lib().o_ppm(_f64(q5), int(step4_as_written), out)
    return out  # qL, qR, dq, q6


def step4(q5):
    """Step 4 detector of one cell from q_{i-2}..q_{i+2}: (eta, hbar)."""
    out = np.zeros(2)
    lib().o_step4(_f64(q5), out)
    return out


def avg(P, y, right_end):
    return lib().o_avg(_f64(P), float(y), int(right_end))


def eigen(rho, p, gam, Bn, Bt1, Bt2):
    R = np.zeros(36); L = np.zeros(36); lam = np.zeros(6); info = np.zeros(9)
    lib().o_eigen(_f64([rho, p, gam, Bn, Bt1, Bt2]), R, L, lam, info)
    keys = ["c", "cf", "cs", "ca", "af", "as", "by", "bz", "sg"]
    return R.reshape(6, 6), L.reshape(6, 6), lam, dict(zip(keys, info))


def face_solve(wl, wr, Bn, stl, str_, tau_h, edge=False, step4_as_written=False):
    out = np.zeros(6)
    lib().o_face_solve(_f64(wl), _f64(wr), float(Bn), _f64(stl).reshape(30), _f64(str_).reshape(30),
                       float(tau_h), int(edge), int(step4_as_written), out)
    return out


def cfl_denominator(rho, v, B, p, gam):
    return lib().o_cfl_denominator(_f64([rho, v[0], v[1], v[2], B[0], B[1], B[2], p, gam]))


def gamma_eff(rho, rh2, rhp=None):
    if rhp is None:
        return lib().o_gamma_eff(float(rho), float(rh2))
    return lib().o_gamma_eff_ions(float(rho), float(rh2), float(rhp))


def temperature(rho, eint, rh2, rhp=0.0):
    """Gas temperature (K) of a cell in code units (rho in m_H cm^-3, rho eps in m_H cm^-3 km^2/s^2)."""
    return lib().o_temperature(float(rho), float(eint), float(rh2), float(rhp))


def ion_rates(T, nH, ne, n):
    """App. D rates of reactions 5-8 and the H+ creation / destruction terms."""
    out = np.zeros(6)
    lib().o_ion_rates(float(T), float(nH), float(ne), float(n), out)
    return dict(zip(["k5", "k6", "k7", "k8", "C", "D"], out))


def run(ic, steps=None, t_end=None, cfl=0.4, **options):
    """Convenience: build a Sim from an initial-condition dict and advance it."""
    nz, ny, nx = ic["rho"].shape
    opts = dict(ic.get("options", {}))
    opts.update(options)
    s = Sim(nx, ny, nz, ic["gamma"], ic["dx"], **opts)
    s.set_state(ic["rho"], ic["mom"], ic["E"], ic["B"], ic.get("rho_h2"))
    if ic.get("rho_hp") is not None:
        s.set_ions(ic["rho_hp"])
    if "bface" in ic:
        s.set_face_B(*ic["bface"])
    if t_end is not None:
        s.advance(cfl, t_end, steps if steps is not None else 1 << 30)
    elif steps:
        for _ in range(steps):
            s.step(cfl)
    return s
