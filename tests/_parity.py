"""Parity bars of the GPU tests (the accuracy target of the build): a returned point must have
relative KKT <= 1e-4 as re-measured by the FP64 oracle, and its objective must agree with the
oracle's tight solve (tol 1e-9, or a stored tol-1e-7 value at the full sizes) to 1e-4
relative."""
REL_KKT = 1e-4
OBJ_REL = 1e-4
TIGHT_TOL = 1e-9


def obj_close(p, pstar, rel=OBJ_REL):
    """|p - p*| <= rel * max(1, |p*|)."""
    return abs(p - pstar) <= rel * max(1.0, abs(pstar))
