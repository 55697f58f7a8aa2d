"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no electronic-structure arithmetic: it only places atoms (bohr), names the
basis-set data files and draws seeded random symmetric matrices.  Both the CPU oracle and the
CUDA library read the same basis files, each with its own parser and normalisation.

Workloads (all coordinates in bohr):
  * ``h2o()``                 one water, O at the origin, O-H 1.809 bohr, H-O-H 104.52 degrees.
  * ``water_cluster(n, box, seed)``  rigid waters, uniform random orientation, O uniform in
                              [0, box]^3, rejection-sampled until every O-O distance >= 5.0 bohr.
  * ``alkane(n, rng)``        linear C_nH_(2n+2) with C-C 2.910, C-H 2.060 bohr, tetrahedral angles
                              and backbone/methyl torsions uniform in [0, 2 pi).
  * ``alkane_batch(count, nmin, nmax, seed)`` a batch of those with n uniform in [nmin, nmax].
  * ``h2(r)``                 H2 on the x axis (the batched dissociation-curve molecule).
"""
from .geometry import (  # noqa: F401
    ATOMIC_NUMBER, SYMBOL, Molecule, h2o, h2, water_cluster, alkane, alkane_batch,
    random_symmetric_density, basis_path,
)
