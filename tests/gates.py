"""Parity bars shared by the GPU tests.

FP64_TOL: the FP64 forms against the FP64 oracle, normwise relative L-inf per
conserved field (both evaluate the same expression forms with IEEE-rounded
FP64 and no contraction, so they agree bit for bit in practice).

MIXED_GATES: the mixed-precision form (FP32 reconstruction, tracing and
Riemann solves; FP64 state, accumulation and dual-energy subtraction) against
the FP64 oracle after the few steps each test runs, normwise relative per
field.  Measured errors sit about ten times below them."""
FP64_TOL = 1e-12
MIXED_GATES = {"linf": 1e-3, "l1": 1e-5}
