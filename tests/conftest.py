import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: long-running (full-size workloads)")
    # the oracle's C part (the multi-core FP64 product) is compiled by the project's build
    # step; it is a no-op when the library is up to date
    import __graft_entry__
    __graft_entry__._build_oracle_c()
