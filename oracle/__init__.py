"""Plain FP64 CPU oracle of the multilevel compressor (TEST INFRASTRUCTURE).

This package is the checker, not the product.  Only the tests, the smoke
check and the benchmark's CPU-baseline / reference legs may import it; the
library path never calls into it and shares no code with it.

The paper (MGARD, "Software design" section) names the pipeline -- recursive
multilevel decomposition of the data into multilevel coefficients on a
multigrid hierarchy, linear quantization of every coefficient to a multiple
of a bin width chosen from the error bound ``tau`` and smoothness ``s``, and
lossless encoding into a self-describing buffer; decompression inverts each
step -- and says the error guarantee comes from finite element theory.  It
prints no formulas.  Each module states the standard P1 finite-element
definitions (nodal hat functions, exact mass matrices, L2 projection) that
the steps rely on, written out as plainly as possible: dense or sparse 1D
matrices applied along one axis at a time.  Readings of points the paper
leaves open are listed in each module's docstring.

Modules
-------
grid        per-dimension node hierarchy (even nodes plus the last node)
fem         1D mass and prolongation matrices on a level's coordinates
multilevel  decompose / recompose (in-place layout), projection norms
bounds      correction-operator norms, bin widths, error norms
quantize    level-wise quantization to dictionary symbols + outliers
huffman     deterministic Huffman code lengths, canonical codes, chunked
            MSB-first bit packing and decoding
pipeline    compress / decompress on top of the above, plus verification
mdr         refactoring: bit-plane segments of every level's coefficients,
            their L-infinity error estimate, greedy plane requests and
            reconstruction
qoi         linear quantities of interest: representer, dual norm and the
            tolerance that bounds a QoI's error
region      region-adaptive L-infinity bounds: far-field tails of the
            correction operators, dilated boxes and per-node widths
ooc         out-of-core blocking along the first axis
predictor   features, MLP and Adam of the learned tolerance predictor

Parity status: every function here is pinned by the CPU tests in
``tests/test_oracle_*.py`` (identities, brute-force dense projections,
closed forms, textbook Huffman costs, exact rational results).
"""
