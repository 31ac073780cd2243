"""Shared parity bookkeeping of the GPU tests.

The error of a result is the plain relative error |a - a_ref| / |a_ref| against the complex128
oracle (or the state vector).  The bounds are those of the workload definition: complex128 1e-12,
complex64 1e-5, TF32 split 1e-5, BF16 split 1e-4.  A bitstring whose reference amplitude is below
1e-3 * 2^(-n/2) -- a thousandth of the typical magnitude of an n-qubit random-circuit amplitude --
is redrawn from the next seed, and the redraw is logged; no other amplitude is excused.

An expectation value <psi|P|psi> of a Pauli string P (for instance Z_i Z_j) is not an amplitude:
its scale is the operator norm ||P|| = 1 that bounds it, not its value, which can be arbitrarily
close to zero.  Its error is therefore measured on that scale, |e - e_ref| / ||P||, against the
same bound (check_observable).  A dense matrix product is checked element by element on the
scale of its largest entry (check_scaled).

Every check records its error under the running test's name; the session prints the largest
error of every test at the end (tests/conftest.py).
"""
import os

import numpy as np

TOL = {"c128": 1e-12, "c64": 1e-5, "tf32": 1e-5, "bf16": 1e-4}
REDRAW_BELOW = 1e-3          # in units of the typical amplitude 2^(-n/2)

MAX_ERR = {}                 # test name -> (largest relative error, its bound)
REDRAWS = []                 # (test name, n, seed tried, |a_ref| / 2^(-n/2))


def _test_name():
    return os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]


def rel_err(got, ref):
    """Plain relative error (|ref| = 0 only when got is exactly 0 too)."""
    got, ref = complex(got), complex(ref)
    if ref == 0:
        return 0.0 if got == 0 else float("inf")
    return abs(got - ref) / abs(ref)


def _record(e, tol):
    name = _test_name()
    old = MAX_ERR.get(name, (0.0, tol))
    MAX_ERR[name] = (max(old[0], e), max(old[1], tol) if old[0] > 0 else tol)


def check(got, ref, tol, what=""):
    """Assert rel_err(got, ref) <= tol and record the error."""
    e = rel_err(got, ref)
    _record(e, tol)
    assert e <= tol, f"{what} relative error {e:.3e} > {tol:.0e} (got {got}, reference {ref})"
    return e


def check_observable(got, ref, tol, norm=1.0, what=""):
    """Expectation value of an observable of operator norm `norm`: |got - ref| / norm <= tol."""
    e = abs(complex(got) - complex(ref)) / norm
    _record(e, tol)
    assert e <= tol, f"{what} error {e:.3e} (on the scale ||P|| = {norm}) > {tol:.0e} (got {got}, reference {ref})"
    return e


def check_scaled(got, ref, scale, tol, what=""):
    """Element-wise |got - ref| / scale <= tol (scale: the largest |entry| of the reference)."""
    e = float(np.max(np.abs(np.asarray(got) - np.asarray(ref)))) / scale
    _record(e, tol)
    assert e <= tol, f"{what} max |error| / scale {e:.3e} > {tol:.0e}"
    return e


def check_all(got, ref, tol, what=""):
    """check() element by element; returns the largest error."""
    got, ref = np.asarray(got).ravel(), np.asarray(ref).ravel()
    worst = 0.0
    for i, (g, r) in enumerate(zip(got, ref)):
        worst = max(worst, check(g, r, tol, f"{what}[{i}]"))
    return worst


def amplitude_bitstring(amp_of, n, seed, draw):
    """A bitstring drawn by draw(n, seed) whose reference amplitude amp_of(x) is at least
    REDRAW_BELOW * 2^(-n/2), trying seed, seed + 1, ...; each redraw is logged.  Returns
    (x, reference amplitude, seed used)."""
    s = seed
    while True:
        x = draw(n, s)
        a = amp_of(x)
        mag = abs(a) / 2.0 ** (-n / 2)
        if mag >= REDRAW_BELOW:
            return x, a, s
        REDRAWS.append((_test_name(), n, s, mag))
        s += 1
