"""FP64 CPU oracle for the CHERT hot path -- TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, obviously correct restatement of what the CUDA
path computes, written from the paper (Darwis et al., "CHERT: Cached
Hamiltonian-Enhanced Ray Tracing in Viscoelastic Anisotropic Media"):

* ``cache_oracle``  -- the directional cache C(m,k,theta) (Eq. 2, 4-7, 9-14, 26,
  35-36): full 4th-order stiffness tensor, Christoffel matrix, numpy
  eigen-decomposition, OEV (Eq. 12) and the literal g*-Hamiltonian form of MEV
  (Eq. 13-14), a brute-force scan of the imaginary slowness angle with
  bisection polish, ray quantities (Eq. 10-11).
* ``graph_oracle``  -- the direction lookup and segment averaging (Eq. 27-30),
  binary-heap Dijkstra for the relaxation fixed point (Eq. 31), the
  deterministic parent rule and raypath backtracking (Eq. 33-34), plus
  Floyd-Warshall for tiny grids.  Dijkstra is plain C (``graph_oracle.c``).
* ``nocache_oracle`` -- the no-cache (MSPM-style) traveltime of the paper's
  Algorithm 1: every node's ray quantities evaluated from its own medium,
  with no table shared between nodes, then the same lookup and Dijkstra.
* ``mlp_oracle`` -- the cache surrogate's network, loss, Adam, BF16 rounding
  and target parametrisation.
* ``coverage_oracle`` -- the nodewise angular-coverage counts (covered stencil
  directions, branch mismatches at folds, missing angles) of one reading of
  the paper's angular-coverage validation.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import or execute anything here.  The product path never does; it
shares no code, header, table or constant generator with this package.

Parity status per function (pins live in ``tests/test_oracle_*.py``):

* moduli_from_thomsen, moduli_from_table -- pinned (Thomsen's forward
  definitions, Table 2 values).
* energy_velocity OEV / MEV, solve_direction, build_cache -- pinned by the
  isotropic closed form, the elastic VTI group velocity, the viscoelastic qSH
  ellipse closed form, Q -> infinity, symmetries, and the paper's printed
  qP imaginary-angle range; MEV away from its real-eigenvector limits is
  **parity unpinned** against the paper (its Eq. 14 is garbled; the reading is
  pinned only to the perturbation-theory identity, not to printed values).
* select_direction, dijkstra, parents, raypath -- pinned by Floyd-Warshall,
  scipy's independent Dijkstra, straight-ray closed forms and reciprocity.
* in_candidates, parent_ties -- pinned by the Manhattan closed form and by
  brute force over Floyd-Warshall distances.
* node_tables, no_cache_fields -- pinned to the cached path (identical
  tables, fields and parents where nodes share a medium).
* coverage_counts, brackets -- pinned by the isotropic closed form,
  hand-built holes, a hand-built fold with known branch velocities, planted
  missing entries, and the convex qP/qSH caches of the layered model.
"""
