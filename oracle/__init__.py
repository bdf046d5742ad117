"""CPU oracle for tiled Householder QR (Bouwmeester, Jacquelin, Langou, Robert,
"Tiled QR factorization algorithms", 2011).

This package is TEST INFRASTRUCTURE.  It is a plain, slow, obviously-correct
restatement of the paper's method, used only to check the CUDA library:

* ``oracle.trees``  -- the elimination lists of every tree (Section 3), the
  validity rules of an elimination list (Section 2.2) and the coarse-grain
  time-step model (Section 3.1).
* ``oracle.dag``    -- expansion of an elimination list into TS or TT kernel
  tasks (Algorithms 2 and 3), their dependencies, and the unit-weight
  as-soon-as-possible simulator that yields zero-out times and critical paths
  (Section 2.3, Table 1 weights).
* ``oracle.kernels`` -- the six FP64 tile kernels (GEQRT, UNMQR, TSQRT, TSMQR,
  TTQRT, TTMQR, Section 2.1) written from the textbook Householder
  definitions, one reflector at a time, plus the compact-WY T factor.
* ``oracle.tiled_qr`` -- the whole tiled factorization run sequentially in
  elimination-list order, and application of Q^T / Q to a right-hand side.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
(``paper_1104_4475_gb300``) and imports nothing from it.

Notation follows the paper: tile rows ``i``, pivot rows ``piv``, panel columns
``k`` and update columns ``j`` are 1-based, a matrix has ``p x q`` tiles of
``nb x nb`` and ``p >= q``.
"""

# Tree identifiers.  The integer values are the same as the library's C enum
# so that a test can name one tree for both sides; nothing else is shared.
FLAT_TS, FLAT_TT, SAMEH_KUCK, BINARY, FIBONACCI, GREEDY, PLASMA, ASAP, GRASAP, PLASMA_TS = range(10)
TREE_NAMES = {
    FLAT_TS: "FlatTree-TS",
    FLAT_TT: "FlatTree-TT",
    SAMEH_KUCK: "Sameh-Kuck",
    BINARY: "BinaryTree",
    FIBONACCI: "Fibonacci",
    GREEDY: "Greedy",
    PLASMA: "PlasmaTree",
    ASAP: "ASAP",
    GRASAP: "GRASAP",
    PLASMA_TS: "PlasmaTree-TS",
}
