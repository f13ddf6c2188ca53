"""CPU FP64 oracle for the symmetric split of a tomographic system.

This package is TEST INFRASTRUCTURE. It is a plain and slow implementation, and
it is meant to be obviously correct. Only three callers may import it:
- the tests,
- the smoke check in ``__graft_entry__``,
- the CPU-baseline leg of ``bench.py``.
The CUDA library never calls it and has no CPU fallback through it.

It shares no code with the CUDA path. The only common inputs are seeded arrays
that the caller passes in.

Citations are to the paper: Alikhanov et al., "About one method of
parallelization of calculations during the reconstruction of a tomographic
image" (arXiv:1902.10559). Equation numbers follow the typeset paper:
- (1) A f = p;
- (2) the symmetry w_{i,j} = w_{M-i+1,N-j+1};
- (3), (4) the two split systems;
- the fold formulas for A and p, which are unnumbered;
- (5) Theorem 1's recombination;
- (12) Theorem 2's recombination;
- (13) Example 1's system;
- (18) the determinant identity.

Modules:
- ``geometry``: symmetric acquisition, vertical-snake numbering, Siddon weights.
  The paper fixes only the symmetry (Section 2, Eq. 2). The ray model follows
  Siddon's exact radiological path.
- ``split``: the fold of A and p, the recombination of Theorem 1 (Eq. 5), the
  image fold from the proof of Theorem 1, and minimum-norm solutions
  (Theorem 2).
- ``sart``: SART-type iteration on the split systems. The simultaneous form
  uses absolute row and column sums.
- ``quant``: BF16/FP16 value storage with per-row scales.
- ``cnn``: the warm-start network's reference forward and backward passes.
"""
