"""Plain FP64 CPU oracle for the superfast line-spectral-estimation hot path.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  It exists to check the CUDA path and
is deliberately slow and obvious: the covariance C is formed as a dense
matrix, factorised by a library Cholesky, and every quantity of the method is
taken from its definition in the paper with dense linear algebra (no
Gohberg-Semencul formula, no Levinson recursion, no FFT, no grid tricks).
It shares no code with the CUDA path.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline`` leg and
``--impl reference``) may import it.

Modules
-------
dense   one evaluation of the model at a state (theta, gamma, beta): C, ln|C|,
        C^{-1}y, the vectors q..x of Sec. II-C, the derivatives, the grid
        quantities and the Gohberg-Semencul generators read off the dense
        inverse.
fit     the block-coordinate-descent estimator of Sec. II (outline in
        Sec. II-D, approximate activation in Sec. II-E), with the
        readings of the paper listed in its docstring.
"""
