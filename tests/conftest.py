import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 (sm_103a) GPU")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    import parity   # tests/ is on sys.path (pytest's prepend import mode), as in the test files
    if parity.MAX_ERR:
        terminalreporter.write_sep("-", "largest relative error per test (plain |a - a_ref| / |a_ref|)")
        for name, (err, tol) in sorted(parity.MAX_ERR.items()):
            terminalreporter.write_line(f"{err:10.3e}  (bound {tol:.0e})  {name}")
    if parity.REDRAWS:
        terminalreporter.write_sep("-", "bitstrings redrawn (|a_ref| below 1e-3 of 2^(-n/2))")
        for name, n, s, mag in parity.REDRAWS:
            terminalreporter.write_line(f"{name}: n={n} seed={s} |a|/2^(-n/2)={mag:.2e}")
