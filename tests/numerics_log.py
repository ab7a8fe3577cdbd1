"""Measured parity figures (largest relative error per test case), collected
by the GPU parity tests and printed in the session summary (tests/conftest.py),
so that a run records the margins, not only pass or fail."""
LOG = []   # (case, quantity, value, tolerance)


def record(case, quantity, value, tol):
    LOG.append((case, quantity, float(value), float(tol)))
    return value
