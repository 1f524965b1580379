"""CPU FP64 oracle for the density-matrix tree approximation (TEST INFRASTRUCTURE).

This package is the plain, slow, obviously-correct restatement of the method used
to check the CUDA path.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import it.  It shares no code with the CUDA
path; the only common dependency is the seeded input generator ``workloads``.

Modules
  exact      plain definitions with exact answers (brute-force spin sums,
             transfer matrices, closed forms, dense network contraction);
             these PIN the method-level code below.
  dmtree     partitioned_contract (Algorithm partitioned_contract, Sec. 3.2)
             over row partitions with the MPS ansatz, calling
             density_matrix_alg (Algorithm density_matrix_alg, Sec. 5) with
             the memoised density matrices of Eq. (dm_cache).
  general    partitioned_contract on arbitrary graphs and partitions (linear
             path, MPS ansatz): edge sets, constraint tree, Kendall-Tau
             ordering, swap passes of Algorithm approx_tensor_network, the
             embedding by minimum cuts, and dmtree's density_matrix_alg on
             the resulting chain blocks.
  canonical  the canonicalisation-based truncation with full environment
             (Sec. 2.2 and Algorithm canonize), an independent algorithm the
             paper states has the same output as the density-matrix one.

Parity status: general is pinned by brute force (chi >= every cut rank, with
and without swap passes), by dmtree at truncating chi (rows as parts), by
embedding independence, and by brute-force checks of its Kendall-Tau and
minimum-cut steps.  dmtree is pinned by exact (chi >= exact rank), by canonical
(chi below exact rank), and by the definition of the density matrix on tiny
networks (Def. density matrix).  Nothing here is "parity unpinned" except
instances whose kept/discarded eigenvalues are (near-)degenerate, where the
kept subspace itself is not unique.
"""
