"""FP64 CPU oracle for the t-product method of Tarzanagh & Michailidis,
"Fast Randomized Algorithms for t-Product Based Tensor Operations and
Decompositions with Applications to Imaging Data" (arXiv 1704.04362).

This package is TEST INFRASTRUCTURE.  It is a plain, slow, obviously correct
restatement of the paper's definitions in NumPy/SciPy float64.  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  The CUDA library never imports, links or calls anything here, and
nothing here imports the CUDA library: the two share no code.

Modules
-------
tensor_ref      Section 2: DFT along mode 3, circ/unfold/fold, the t-product
                (Def. 2.1, Algorithm 1), conjugate transpose, identity tensor,
                norms (Def. 2.7, tensor nuclear norm).
philox_ref      Philox4x32-10 counter-based generator (Salmon et al., SC'11)
                and the integer Bernoulli decision used for slice draws.
sampling_ref    Section 3.1: slice norms, sampling probabilities (eqs. for the
                "nearly optimal" and "A-only" choices), Algorithm 2
                (rt-product).
learned_ref     Per-frequency adaptive rank rule for the randomized t-SVD and
                the rank/oversampling predictor network (features, forward,
                back-propagation, Adam): not in the paper; it fixes what the
                predictor kernels compute.
decomp_ref      Theorem 2.6 (t-SVD by facewise SVD), randomized low-tubal-rank
                t-SVD (Halko-Martinsson-Tropp range finder per frequency),
                Algorithm 3/4 (t-project, t-CX).
completion_ref  Appendix Algorithm 7 (ADMM) in its tensor-completion form of
                problem (tlow6), with tensor singular-value thresholding.

Parity status: every function is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (identities, closed forms, brute force, library
special cases).  Functions without such a pin are marked "parity unpinned"
in their docstring; there are none at present.
"""
