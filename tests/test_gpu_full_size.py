"""The two full-size J/K workloads against the FP64 CPU oracle, in the launch configuration the
benchmark times: kernel choice autotuned per bin part, then the device-pointer build.

  (H2O)_8  / 6-31G*, seed 2002, 12-bohr cube:  152 functions
  (H2O)_32 / 6-31G*, seed 2006, 19-bohr cube:  608 functions
  Schwarz threshold 1e-10 (the same rule, Q_ab Q_cd >= tau, on both sides).

Sampled J/K elements are compared with the oracle's defining sums over all (l, s) - FP64 within
1e-8, the reduced-precision form within 2e-5 per element - covering O-d/O-d, O-s/H-s and diagonal
elements.  The reduced-precision energy bar (|dE| <= 1e-6 Ha) is checked on a converged density
against the FP64 build, which the sampled elements hold to the oracle."""
import numpy as np
import pytest
import torch

import mess_inputs as mi
from gpu_helpers import converged_density, sample_pairs

pytestmark = pytest.mark.gpu

TAU = 1e-10
FP64_TOL = 1e-8          # max |dJ|, |dK| of the FP64 path
MIXED_ELEM_TOL = 2e-5    # per element, reduced-precision path (FP32 recursion)
ENERGY_TOL = 1e-6        # |dE| of the reduced-precision path, Ha

WORKLOADS = {
    "water8": dict(n=8, box=12.0, seed=2002, nbf=152, per_kind=24, n_random=8),
    "water32": dict(n=32, box=19.0, seed=2006, nbf=608, per_kind=12, n_random=4),
}
MIXED = dict(prec="mixed", schwarz_tau=TAU, split_df32=True)
FP64 = dict(prec="fp64", schwarz_tau=TAU)


def _device_build(g, D, **kw):
    """The benchmark's call: device buffers, the caller's stream, synchronised here."""
    dev = torch.device("cuda", 0)
    dD = torch.from_numpy(np.ascontiguousarray(D)).to(dev)
    dJ, dK = torch.empty_like(dD), torch.empty_like(dD)
    s = torch.cuda.current_stream(dev)
    info = g.jk_device(dD, dJ, dK, stream=s, **kw)
    torch.cuda.synchronize(dev)
    return dJ.cpu().numpy(), dK.cpu().numpy(), info


@pytest.fixture(scope="module", params=sorted(WORKLOADS))
def workload(request, mess, oracle_mod):
    w = WORKLOADS[request.param]
    mol = mi.water_cluster(w["n"], w["box"], w["seed"])
    path = mi.basis_path("6-31gs")
    g = mess.Basis.from_molecule(mol, path)
    o = oracle_mod.basis_for(mol, path)
    assert g.nbf == o.nfn == w["nbf"]
    return request.param, w, g, o


def test_sampled_elements_fp64_and_mixed(workload, oracle_mod):
    name, w, g, o = workload
    D = mi.random_symmetric_density(g.nbf, w["seed"])
    rows, cols = sample_pairs(o, np.random.default_rng(w["seed"]), w["per_kind"], w["n_random"])
    assert len(rows) >= (64 if name == "water8" else 32)
    Jr, Kr = oracle_mod.jk_elements(o, D, rows, cols, tau=TAU, Q=oracle_mod.schwarz(o))
    for kw, tol in ((FP64, FP64_TOL), (MIXED, MIXED_ELEM_TOL)):
        g.jk_autotune(D, reps=1, **kw)
        J, K, info = _device_build(g, D, **kw)
        dj = np.abs(J[rows, cols] - Jr).max()
        dk = np.abs(K[rows, cols] - Kr).max()
        print(f"{name} {kw['prec']}: {len(rows)} elements, max|dJ| = {dj:.2e}, max|dK| = {dk:.2e}")
        assert dj <= tol and dk <= tol, (kw["prec"], dj, dk)
        assert np.array_equal(J, J.T) and np.array_equal(K, K.T)
        assert info["shell_quartets"] > 0
        if kw["prec"] == "mixed":
            assert 0 < info["shell_quartets_fp64"] < info["shell_quartets"]


def test_mixed_energy_error_on_converged_density(workload):
    """E_2(D) = 1/2 sum D (J - K/2) of the reduced-precision build against the FP64 build, both on
    the same converged density, with the Boys function in FP32 (default) and in FP64."""
    name, w, g, o = workload
    D = converged_density(g, schwarz_tau=TAU)
    e2 = lambda J, K: 0.5 * float(np.sum(D * (J - 0.5 * K)))  # noqa: E731
    J64, K64, _ = _device_build(g, D, **FP64)
    for boys64 in (False, True):
        J, K, _ = _device_build(g, D, boys_fp64=boys64, **MIXED)
        dE = e2(J, K) - e2(J64, K64)
        print(f"{name} mixed (boys_fp64={boys64}): dE = {dE:.3e} Ha")
        assert abs(dE) <= ENERGY_TOL, (boys64, dE)
