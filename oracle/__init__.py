"""CPU oracle of the counter-guided search step (arXiv 2102.05297).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the method, written from the paper's Sections 3.3-3.6 and
Algorithm 1.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it.  It shares no code with the CUDA library
(``paper_2102_05297_gb300``) and never imports it; both sides read only the
seeded inputs of ``workloads``.

Floating point: every quantity the paper defines is computed in float64 (the
"definition"); where a float result decides an integer (the quantised
selection weights, the top-k order) the oracle also offers the float32 path in
the same operation order as the kernels, so that both sides take the decision
in the same precision.

Modules
  space    Section 1 / Algorithm 1 input TS: mixed-radix decode, constraint
           bytecode, enumeration of the valid space.
  trees    Section 3.3.2: regression-tree prediction (pointer walk) and a
           plain CART fitter.
  expert   Section 3.4: bottleneck analysis (B) and the Delta-PC reaction.
  score    Section 3.5, Eq. "score".
  select   Section 3.5 Eq. "score_normalization", Section 3.6 / Algorithm 1
           weighted draws; Philox4x32-10 counter-based generator; top-k.
  search   Algorithm 1 end to end.
  mlp      the learned surrogate (BF16 rounding points, FP32 accumulate).
  lsq      Section 3.3.1: least-squares regression per binary-parameter subspace.
  nbr      steps restricted to c_profile's Hamming neighbourhood (Section 3.5
           footnote; local search, Section 3.8.1).

Parity status of each function is stated in its docstring; the only unpinned
part is the heuristic's selected set beyond its own definition.
"""
