"""mess_jk_build_static: the J/K build for callers that cannot let the library allocate device memory
(their device memory belongs to their own pool, or cudaFree's implicit synchronisation is not
acceptable on their path).  It stages D, J and K in a fixed array inside the library, so its results
must equal those of mess_jk_build, which allocates its staging buffers per call.

The file is named to be collected last; every test here goes through the C ABI (the ctypes
functions of the binding) and works in a fresh process as well as after the other tests."""
import ctypes

import numpy as np
import pytest

import mess_inputs as mi

pytestmark = pytest.mark.gpu

TOL = 1e-8   # the FP64 J/K parity tolerance of the other GPU tests


def _call(fn, mess, g, D, opts):
    n = g.nbf
    D = np.ascontiguousarray(D, dtype=np.float64)
    J, K = np.zeros((n, n)), np.zeros((n, n))
    info = mess.mess_jk_info()
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
    st = fn(g.handle, dp(D), dp(J), dp(K), ctypes.byref(opts), ctypes.byref(info))
    return st, J, K


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_static_matches_allocating_build_on_two_calls(mess, prec):
    g = mess.Basis.from_molecule(mi.water_cluster(2, 9.0, 11), mi.basis_path("6-31gs"))
    opts = mess.jk_opts(prec, schwarz_tau=1e-10)
    densities = [mi.random_symmetric_density(g.nbf, seed) for seed in (5, 6)]
    refs = []
    for D in densities:
        st, J, K = _call(mess.mess_jk_build, mess, g, D, opts)
        assert st == mess.MESS_OK
        refs.append((J, K))
    # two calls in a row: the second must not see the first call's staged contents
    for D, (Jr, Kr) in zip(densities, refs):
        st, J, K = _call(mess.mess_jk_build_static, mess, g, D, opts)
        assert st == mess.MESS_OK, mess.mess_last_error()
        assert np.abs(J - Jr).max() <= TOL
        assert np.abs(K - Kr).max() <= TOL


def test_static_rejects_what_it_cannot_do_without_allocating(mess):
    # bins for new options do not exist yet: building them would allocate
    g = mess.Basis.from_molecule(mi.h2o(), mi.basis_path("sto-3g"))
    D = mi.random_symmetric_density(g.nbf, 1)
    st, _, _ = _call(mess.mess_jk_build_static, mess, g, D, mess.jk_opts("fp64", schwarz_tau=1e-9))
    assert st == mess.MESS_EINVAL
    assert b"bins" in mess.mess_last_error()
    # more functions than the static workspace holds
    big = mess.Basis.from_molecule(mi.water_cluster(14, 22.0, 3), mi.basis_path("6-31gs"))
    assert big.nbf > 256
    st, _, _ = _call(mess.mess_jk_build_static, mess, big, np.eye(big.nbf), mess.jk_opts("fp64"))
    assert st == mess.MESS_EINVAL
    assert b"256" in mess.mess_last_error()
