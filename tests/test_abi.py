"""The C-ABI library builds for sm_103a, loads, and exports every entry point
``include/imblbm.h`` declares.  No compute call is made (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "imblbm.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(imb3?_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1809_07008_gb300 import binding
    return binding.load()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("imb_init_lattice", "imb_set_particles", "imb_step", "imb_get_populations",
              "imb_get_macro", "imb_get_forces", "imb_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1809_07008_gb300 import binding
    out = subprocess.run(["nm", "-D", "--defined-only", binding.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\b(imb3?_\w+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    assert sorted(binding.EXPORTS) == _declared()
    for n in _declared():
        assert isinstance(getattr(lib, n), ctypes._CFuncPtr)


def test_default_params_match_header(lib):
    from paper_1809_07008_gb300 import binding
    p = binding.default_params()
    assert (p.bc_x, p.bc_y, p.storage, p.eps_mode, p.n_sub) == (0, 1, 0, 0, 5)
    assert (p.N_sub, p.kn, p.kt, p.e_rest, p.mu, p.rho_s, p.skin) == (100, 1e5, 5e4, 0.5, 0.5, 2.65, 1.0)
    assert p.rho0 == 1.0 and p.timeout_ms == 60000


def test_params_struct_layout_matches_header(lib):
    # the ctypes mirror must list the header's fields in the same order
    from paper_1809_07008_gb300 import binding
    txt = open(HEADER).read()
    body = txt[txt.index("typedef struct imb_params {"):txt.index("} imb_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in re.findall(r"(int|double)\s+([^;]+);", body):
        fields += [f.strip() for f in decl[1].split(",")]
    assert [f[0] for f in binding.Params._fields_] == fields


def test_params3_struct_layout_matches_header(lib):
    from paper_1809_07008_gb300 import binding
    txt = open(HEADER).read()
    body = txt[txt.index("typedef struct imb3_params {"):txt.index("} imb3_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in re.findall(r"(int|double)\s+([^;]+);", body):
        fields += [f.strip() for f in decl[1].split(",")]
    assert [f[0] for f in binding.Params3._fields_] == fields
    p = binding.Params3()
    lib.imb3_default_params(ctypes.byref(p))
    assert (p.wall_y, p.n_sub, p.storage, p.rho0, p.timeout_ms) == (1, 5, 0, 1.0, 60000)
