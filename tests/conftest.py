import os
import sys

# The FP64 oracle works on many small dense blocks: one BLAS thread is the
# fastest setting for it, and several threads on a shared host contend badly
# (a 512 x 512 oracle factorization took minutes instead of ~25 s).  Set
# before numpy is first imported.
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import pytest  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the built library")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")
