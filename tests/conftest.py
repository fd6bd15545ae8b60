import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


# With GBS_ERRLOG=<path>, every oracle.err_norms call made by a test appends
# one JSON line (the test's node id and the norms) to <path>: the record from
# which the multi-step tolerance is fitted.  Off by default.
_ERRLOG = os.environ.get("GBS_ERRLOG")
if _ERRLOG:
    import json

    import oracle as _oracle

    _err_norms = _oracle.err_norms

    def _logged_err_norms(*args, **kwargs):
        e = _err_norms(*args, **kwargs)
        rec = {"test": os.environ.get("PYTEST_CURRENT_TEST", "")}
        for k, v in e.items():
            try:
                rec[k] = float(v)
            except (TypeError, ValueError):
                rec[k] = str(v)
        with open(_ERRLOG, "a") as f:
            f.write(json.dumps(rec) + "\n")
        return e

    _oracle.err_norms = _logged_err_norms
