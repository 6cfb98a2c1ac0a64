"""CPU oracle for the pruning + domain-selection Ising solver.

Plain, slow, obviously correct FP64 (or exact integer) restatement of
Li, Dong and Pan, "Fast Numerical Solver of Ising Optimization Problems via
Pruning and Domain Selection": Sec. II (energy), Sec. III-A / Algorithm 1
(pruning), Sec. III-B (domain selection, Eq. loss function) and Sec. IV
(metrics: pruning rate, Hamiltonian ratio, time-to-solution, speed).

THIS PACKAGE IS TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it. The CUDA library shares no code with it and never calls it; the product
path fails loudly when its compiled library is missing instead of falling back
here.

Modules and what pins them (tests marked ``not gpu``):

* ``ising``            energy three ways, single-flip difference, max-cut value.
                       Pinned: the three forms agree exactly on integer
                       instances, the single-flip identity of Sec. III-A against
                       re-evaluation, cut(s) = W/2 - E(s) for J = -W/2 against
                       edge counting.
* ``rng``              SplitMix64 counter generator (Steele, Lea, Flood 2014).
                       Pinned: published first outputs for seed 0.
* ``domain_selection`` the relaxed gradient-descent step and the restart loop.
                       Pinned: gradient against central finite differences of
                       the loss with the rounded spins frozen; Adam update
                       against torch.optim.Adam (fp64, CPU); first-step
                       |delta theta| = lr; brute-force ground states reached on
                       small instances; best tracking against the recorded
                       energy trace. The per-step trajectory itself has no
                       worked example in the paper (parity of the update rule
                       rests on these identities).
* ``pruning``          Algorithm 1 with the readings listed in its docstring,
                       and reconstruction. Pinned: brute-force minima for
                       n <= 16 (pruning is exact), E_full(reconstruct(s_G)) =
                       E_G(s_G) + C, zero field reduces to 2-core peeling
                       (networkx.k_core), Binary family prunes nothing, the
                       first-round rate closed form and the Table 1 pruning
                       rates.
* ``brute_force``      exhaustive minimum for n <= 20 (vectorised enumeration).
                       Pinned: hand-solvable cases (ferromagnet, single bond,
                       frustrated triangle).
* ``metrics``          pruning rate, Hamiltonian ratio, TTS, speed, first-round
                       estimate. Pinned: Table 2 rows (T, chi_hat -> TTS, v) and
                       the first-round closed form for the uniform family.
"""

from . import ising, rng, domain_selection, pruning, brute_force, metrics  # noqa: F401
