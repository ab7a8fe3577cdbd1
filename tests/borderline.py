"""Encounter decisions close to the critical radius.

A candidate pair whose separation lies within 1e-12 relative of its critical
radius rc_ij (before or after the drift) is one where a rounding difference in
the state could flip the detection decision.  The parity tests collect such
pairs here; the session summary prints them (tests/conftest.py)."""
import numpy as np

REL = 1e-12
LOG = []          # (case, candidates, [(tag, i, j, |r/rc_ij - 1|), ...])


def near_critical(cand, x1, x2, rc, rel=REL):
    cand = np.asarray(cand, dtype=np.int64).reshape(-1, 2)
    i, j = cand[:, 0], cand[:, 1]
    rcij = np.maximum(rc[i], rc[j])
    out = []
    for tag, x in (("pre-drift", x1), ("post-drift", x2)):
        d = x[j] - x[i]
        r = np.sqrt((d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2])
        q = np.abs(r / rcij - 1.0)
        for k in np.nonzero(q <= rel)[0]:
            out.append((tag, int(i[k]), int(j[k]), float(q[k])))
    return out


def record(case, cand, x1, x2, rc):
    found = near_critical(cand, x1, x2, rc)
    LOG.append((case, len(cand), found))
    return found
