"""The C-ABI library builds for sm_103a, loads, and exports every entry point
``include/imblbm.h`` declares; the parameter structs mirror the header; and the host-side
argument checks (which run before any CUDA call) refuse bad sizes, relaxation times,
Smagorinsky constants, disks and oversized launches.  No compute call is made (no GPU needed)."""
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
    assert p.rho0 == 1.0 and p.timeout_ms == 60000 and p.work_units == 0 and p.plain_launches == 0


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


def test_host_validation_refuses_before_any_device_call(lib):
    # the argument checks of imb3_init, imb_init_lattice and imb_batch_create run on the host
    # before the first CUDA call, so their refusals answer here without a GPU
    import numpy as np
    from paper_1809_07008_gb300 import binding as B
    C = ctypes
    BAD = -1   # IMB_E_INVALID_ARG
    h = C.c_void_p()
    p3 = B.Params3()
    lib.imb3_default_params(C.byref(p3))
    assert p3.C_smag == 0.0 and p3.n_sub == 5
    assert lib.imb3_init(C.byref(h), 2, 10, 10, 0.8, C.byref(p3)) == BAD and not h.value
    assert lib.imb3_init(C.byref(h), 10, 10, 10, 0.5, C.byref(p3)) == BAD
    p3.C_smag = -0.1
    assert lib.imb3_init(C.byref(h), 10, 10, 10, 0.8, C.byref(p3)) == BAD and not h.value
    assert b"C_smag" in lib.imb3_last_error(None)
    p3.C_smag, p3.n_sub = 0.0, 11
    assert lib.imb3_init(C.byref(h), 10, 10, 10, 0.8, C.byref(p3)) == BAD
    p = B.default_params()
    assert lib.imb_init_lattice(C.byref(h), 64, 32, 0.6, -0.1, C.byref(p)) == BAD and not h.value
    assert lib.imb_init_lattice(C.byref(h), 64, 32, 0.5, 0.0, C.byref(p)) == BAD

    def batch(nx, ny, tau, xy, r):
        n = len(r)
        ints = lambda v: np.array([v], dtype=np.int32)
        dbl = lambda v: np.array([v], dtype=np.float64)
        hb = C.c_void_p()
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1)
        r = np.ascontiguousarray(r, dtype=np.float64)
        rc = lib.imb_batch_create(C.byref(hb), 1, ints(nx).ctypes.data_as(B._ip), ints(ny).ctypes.data_as(B._ip),
                                  B._d(dbl(tau)), B._d(dbl(0.0)), B._d(dbl(1e-6)), B._d(dbl(0.0)),
                                  ints(n).ctypes.data_as(B._ip), B._d(xy), B._d(r), 0)
        assert not hb.value
        return rc

    assert batch(128, 128, 0.5, [[64.0, 64.0]], [5.0]) == BAD              # tau <= 1/2
    assert batch(128, 128, 0.6, [[130.0, 64.0]], [5.0]) == BAD             # centre outside
    assert batch(128, 128, 0.6, [[64.0, 64.0]], [62.5]) == BAD             # wider than the domain - 4
    # 20 000 disks of radius 2046 in one 4096^2 domain pass every per-disk check, but their
    # solid-ratio launch would need 20 000 x 4095^2 / 128 > 2^31 - 1 blocks
    n = 20000
    assert batch(4096, 4096, 0.6, np.full((n, 2), 2048.0), np.full(n, 2046.0)) == BAD


def test_step_io_marshalling_passes_each_arrays_own_address():
    # the per-cycle call's marshalling, with the library call replaced by a recorder: every
    # pointer argument is the data address of the array given for it (looked up once per array
    # object, so an array freed and another allocated in its place, possibly under the same id,
    # gets its own address), non-contiguous or non-float64 inputs go as converted copies that
    # hold the same values, and malformed outputs are refused before the call
    import numpy as np
    from paper_1809_07008_gb300 import binding

    calls = []

    class Recorder:
        def imb_step_io(self, h, n, *ptrs):
            # the arrays behind the addresses, read while the call is in progress
            calls.append((n, ptrs))
            return 0

    class Host:
        np = 5
        h = None
        _L = Recorder()
        _io_addr = binding.Lattice._io_addr

        def __init__(self):
            self._addr_table = {}

        def _check(self, rc):
            assert rc == 0

    lat = Host()
    n = Host.np

    def arrays():
        return (np.arange(2 * n, dtype=np.float64).reshape(n, 2), np.ones((n, 2)), np.zeros(n),
                np.zeros((n, 2)), np.zeros(n))

    for rnd in range(3):
        x, v, w, F, T = arrays()
        binding.Lattice.step_io(lat, 2, (x, v, w), F, T, x, v, w)
        got = calls[-1][1]
        want = [a.ctypes.data for a in (x, v, w, F, T, x, v, w)]
        assert calls[-1][0] == 2 and list(got) == want, rnd
        del x, v, w, F, T   # the next round's arrays may reuse these ids and addresses

    x, v, w, F, T = arrays()
    vf = np.asfortranarray(np.stack([np.arange(n, dtype=np.float64), -np.arange(n, dtype=np.float64)], axis=1))
    seen = {}

    class Reader(Recorder):
        def imb_step_io(self, h, n_, *ptrs):
            # the converted velocity copy, read back from its address during the call
            buf = (ctypes.c_double * (2 * n)).from_address(ptrs[1])
            seen["v"] = np.frombuffer(buf, dtype=np.float64).copy()
            return 0

    lat._L = Reader()
    binding.Lattice.step_io(lat, 1, (x, vf, w.astype(np.float32)), F, T)
    assert np.array_equal(seen["v"], np.ascontiguousarray(vf).reshape(-1))
    lat._L = Recorder()
    binding.Lattice.step_io(lat, 1)
    assert calls[-1][1] == (None,) * 8
    for bad in (np.zeros((n, 2), dtype=np.float32), np.zeros((n, 3)), np.zeros((2, n)).T, [0.0] * (2 * n)):
        with pytest.raises(ValueError):
            binding.Lattice.step_io(lat, 1, None, bad)
    for kin in ((x, v), (x, v, w, w)):
        with pytest.raises(ValueError):
            binding.Lattice.step_io(lat, 1, kin)
