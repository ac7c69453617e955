"""The bounds-checked build (SNN_CHECK: every record's target and delay,
every tile index entry and the order of every list's chunk offsets checked
before use) run over the small parity cases: a child process loads
libsnn_check.so (SNN_CHECKED=1), runs the delivery, update, simulation,
partition and STDP parity tests plus the corrupted-store test, and then no
net of the clean cases may have raised SNN_ERRF_CHECK."""
import os
import subprocess
import sys

import pytest

from gpu_common import need_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CLEAN = ["tests/test_gpu_deliver.py", "tests/test_gpu_update.py",
         "tests/test_gpu_simulate.py", "tests/test_gpu_partition.py",
         "tests/test_gpu_stdp.py"]

_CHILD = """
import sys
import pytest
rc = pytest.main(["-x", "-q", "-m", "gpu", "-p", "no:cacheprovider", *sys.argv[1:]])
from paper_2109_12855_gb300 import snn
assert snn.snn_checked()
n = snn.snn_debug_check_failures()
print("nets flagged by the bounds checks:", n)
sys.exit(rc if rc else (3 if n else 0))
"""


def _run(files):
    env = dict(os.environ, SNN_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", _CHILD, *files], cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=1800)
    return r.returncode, r.stdout[-3000:] + r.stderr[-2000:]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def test_clean_parity_cases_raise_no_check():
    rc, out = _run(CLEAN)
    assert rc == 0, out
    assert "nets flagged by the bounds checks: 0" in out


def test_corrupt_store_is_caught_by_the_checks():
    rc, out = _run(["tests/test_gpu_checked_store.py"])
    # every corrupted net is flagged (and counted): exit status 3, tests green
    assert rc == 3, out
    assert "5 passed" in out, out
