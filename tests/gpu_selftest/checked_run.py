"""Child process of tests/test_gpu_checked_build.py: runs the step paths on small, ragged and
degenerate boxes with the index-checked library (libmhd_check.so) and prints its check flags."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1608_08748_gb300 import build as B  # noqa: E402

B.LIB = B.build(check=True)  # the binding loads the checked library in this process
import ctypes  # noqa: E402

import paper_1608_08748_gb300 as M  # noqa: E402
from paper_1608_08748_gb300 import inputs as I  # noqa: E402

L = M.lib()
L.mhd_check_flags.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_uint)]
flags = ctypes.c_uint(0)
assert L.mhd_check_flags(1, ctypes.byref(flags)) == 0  # a checked library answers

shapes = [(5, 7, 9), (17, 9, 5), (1, 1, 16), (2, 3, 1), (33, 8, 12)]
runs = 0
for precision in (0, 1):
    for k, shape in enumerate(shapes):
        for bc in [(0, 0, 0), (1, 1, 1), (1, 0, 1)]:
            ic = I.turbulence(8, mach=3.0, seed=40 + k, shape=shape)
            ic["options"] = dict(ic["options"], bc_x=bc[0], bc_y=bc[1], bc_z=bc[2])
            s = M.from_ic(ic, precision=precision)
            for _ in range(2):
                s.step(0.4)
            s.get_state()
            s.diagnostics()
            runs += 1
    sims = [M.from_ic(I.turbulence(8, mach=2.0, seed=60 + k, shape=sh), precision=precision)
            for k, sh in enumerate([(8, 16, 24), (9, 10, 11), (16, 8, 8)])]
    b = M.Batch(sims)
    for _ in range(2):
        b.step(0.4)
    b.sync()
    b.close()
    runs += 1
g = M.from_ic(I.turbulence(8, mach=2.0, seed=70, shape=(12, 10, 8)), grav_g=1e-4)  # Poisson kernels
g.step(0.4)
ions = I.turbulence(8, mach=2.0, seed=71, shape=(7, 9, 11))
ions["rho_h2"] = 0.05 * ions["rho"]
ions["rho_hp"] = 1e-3 * ions["rho"]
h = M.from_ic(ions, heatcool=1, ions=1)
h.step(0.4)
assert L.mhd_check_flags(0, ctypes.byref(flags)) == 0
print(json.dumps({"runs": runs + 2, "flags": int(flags.value)}))
