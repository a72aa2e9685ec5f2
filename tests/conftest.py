import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")


def rel_l2(a, b):
    import numpy as np
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


# Parity tolerances.  Relative L2 over the whole output is the accuracy target
# (FP64-class plans 1e-10, FP32-class plans 1e-5).  The element-wise bound is
# max |got - ref| / rms(ref): it catches an error confined to a few samples
# (a pole, a ghost row, a tile edge) that the global norm would average away.
# Measured worst cases: FP64 1.5e-12 and DF64 3.4e-12 (adjoint cubes and
# gradients), FP32 4.7e-6, the 3xTF32 tensor-core contraction 2.4e-5 (its cube
# carries ~5x the FP32 error); each bound leaves a margin of 3-5x.
TOL64, TOL32 = 1e-10, 1e-5
MAX64, MAX32, MAXTC = 1e-11, 2e-5, 1e-4


def rms(a):
    import numpy as np
    a = np.asarray(a)
    return float(np.sqrt(np.mean(np.abs(a) ** 2)))


def check_close(got, ref, l2_tol, max_tol, label=""):
    """Assert relative L2 < l2_tol and max|got - ref| / rms(ref) < max_tol;
    print both and return them."""
    import numpy as np
    got, ref = np.asarray(got), np.asarray(ref)
    assert got.shape == ref.shape, (label, got.shape, ref.shape)
    e2 = rel_l2(got, ref)
    em = float(np.max(np.abs(got - ref))) / max(rms(ref), 1e-300) if ref.size else 0.0
    print("%s: rel L2 %.2e, max|err|/rms %.2e" % (label, e2, em))
    assert np.all(np.isfinite(got)), (label, "non-finite output")
    assert e2 < l2_tol and em < max_tol, (label, e2, em, l2_tol, max_tol)
    return e2, em


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle
