"""FP64 CPU oracle for the FourierSMT hot path (arxiv 2603.22877).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
baseline leg of the benchmark may import this package.  The product path (the
CUDA library and its Python binding) never imports, calls or links it, and the
oracle imports nothing from the product package: the two share no code.  Both
consume the seeded inputs of the separate ``workloads`` package.

Modules
  bdd        reduced ordered BDDs built with Bryant's apply over each
             constraint's literal order (Suppl. Note "Decision Diagrams",
             Def. xBDD: atoms are treated as propositional variables)
  semantics  the Boolean function of each constraint kind and the exact
             (rational) truth value of an atom
  relax      randomized rounding (Eq. rounding) and Gaussian smoothing
             (Eq. sampling) with the derivative of d_i(b)
  cop        COP by its definition (sum over all literal assignments) and by
             the forward / backward message passing of Alg. 3 / Alg. 4
  objective  C_sigma(a, b) = sum_c w_c (1 - 2 COP_c) and its exact gradient
  pgd        projection (Def. Projection / Prop. QP), the projected gradient
             mapping (Eq. grad_map), the epsilon stopping rule, rounding and the
             exact check (Alg. 1), and annealing with ERWA weights (Alg. 2)

Pinning status (what fixes each function independently of itself) is listed in
each module's docstring.  Functions without an independent pin say
"parity unpinned".
"""
