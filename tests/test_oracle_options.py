"""The oracle wrapper's option keys equal the numbering of the oracle's C enum, and every option is
accepted with a valid value and rejected with an invalid one (where one exists)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def c_enum():
    src = open(os.path.join(ROOT, "oracle", "mhd_oracle.c")).read()
    body = re.search(r"enum \{\s*(O_BC_X.*?)\};", src, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    return {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"O_([A-Z0-9_]+)\s*=\s*(\d+)", body)}


def test_wrapper_keys_equal_the_c_enum(oracle_mod):
    assert oracle_mod.OPT == c_enum()


@pytest.mark.parametrize("key,good,bad", [("bc_x", 1, 2), ("regul_mode", 2, 3), ("heatcool", 1, 2),
                                          ("ions", 1, 2), ("chem_bdop", 3.0, 0.0), ("grav_g", 1e-4, -1.0)])
def test_options_validate(oracle_mod, key, good, bad):
    s = oracle_mod.Sim(4, 4, 4, 5.0 / 3.0, 1.0)
    s.set_option(key, good)
    with pytest.raises(ValueError):
        s.set_option(key, bad)
