"""The C-ABI library loads and exports every entry point include/mess.h declares (no GPU needed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mess.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mess_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("mess_basis_create", "mess_overlap", "mess_kinetic", "mess_nuclear", "mess_jk_build",
                     "mess_jk_build_device", "mess_scf", "mess_nuclear_repulsion", "mess_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from conftest import build_library
    lib_path = build_library()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(mess):
    m = mess
    assert sorted(m.EXPORTED) == _declared()
    for n in _declared():
        assert callable(getattr(m, n))


def test_invalid_arguments_are_rejected_without_a_gpu(mess):
    m = mess
    h = ctypes.c_void_p()
    st = m.mess_basis_create(0, None, None, b"nofile", ctypes.byref(h))
    assert st == m.MESS_EINVAL
    assert b"bad structure" in m.mess_last_error()
    assert m.mess_basis_nbf(None) == -1
    m.mess_basis_destroy(None)


def test_basis_creation_needs_no_gpu(mess):
    """Creating a basis reads the basis file and expands the shells on the host only (the device
    data is built by the first computation), so its sizes are available without a GPU."""
    import mess_inputs as mi
    g = mess.Basis.from_molecule(mi.h2o(), mi.basis_path("6-31gs"))
    assert (g.nbf, g.nshell, g.nelectron) == (19, 10, 10)     # O: 1s 2s 2p 3s 3p d = 15; H: 2 x 2
    # O-H 1.809 bohr twice, H-H 2 x 1.809 sin(52.26 deg)
    import math
    e = 2 * 8.0 / 1.809 + 1.0 / (2 * 1.809 * math.sin(math.radians(52.26)))
    assert abs(g.nuclear_repulsion() - e) < 1e-12 * e
    a = mess.Basis.from_molecule(mi.alkane(3, __import__("numpy").random.default_rng(1)), mi.basis_path("sto-3g"))
    assert a.nbf == 7 * 3 + 2 and a.nelectron == 26
    g.close()
    a.close()
