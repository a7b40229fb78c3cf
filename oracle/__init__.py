"""Oracle: plain, slow FP64 CPU implementation of one-way-QC pattern
simulation, written from the paper.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check in
__graft_entry__ and the CPU-baseline leg of bench.py may import or run it; the
product library never does.  It shares no code with the CUDA path: the only
common module is the seeded input generator package `owqs_inputs`.

Contents
  basis      measurement basis |+-a>, operators M0/M1/P0/P1 (Eqs. 1, 9-12),
             signal-dependent angle (Eq. 2), well-formedness D0-D3 (Sec. 2.2)
  substate   O-A: sub-state simulator with qubit elimination (Secs. 4.1-4.4)
  brute      O-B: full-register simulator with projectors, no elimination
             and no reordering (Eqs. 3-4, 9-10)
  proa       greedy pattern reordering with the Eq. 18 cost (Sec. 4.3)
  circuit    textbook J(alpha)/CZ circuit unitaries (dense matrix products)
  counting   amplitude-update count of a command sequence

Parity status: every function is pinned by tests/test_oracle_pins.py against
values the paper prints (Figure 8, Table I, Eqs. 8, 21-23), closed forms
(J(alpha), CZ, CNOT, J/CZ circuit products), invariants (norm, probability
sums, determinism of flow patterns, independence of the command order) and
brute force (O-A against O-B).
"""
