import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long CPU check, run with POSIT_SLOW=1")


def pytest_collection_modifyitems(config, items):
    if os.environ.get("POSIT_SLOW") == "1":
        return
    skip = pytest.mark.skip(reason="slow check; set POSIT_SLOW=1")
    for it in items:
        if "slow" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(scope="session")
def posit_checker(tmp_path_factory):
    """Compile tests/c/posit_check.c against the oracle library."""
    import oracle
    libpath = oracle.build()
    libdir = os.path.dirname(libpath)
    out = tmp_path_factory.mktemp("checker") / "posit_check"
    src = os.path.join(ROOT, "tests", "c", "posit_check.c")
    subprocess.run(["gcc", "-O2", "-fopenmp", "-std=gnu11", "-o", str(out), src,
                    f"-L{libdir}", "-loracle", f"-Wl,-rpath,{libdir}", "-lm"],
                   check=True)

    def run(*args):
        r = subprocess.run([str(out)] + [str(a) for a in args],
                           capture_output=True, text=True)
        line = [ln for ln in r.stdout.splitlines() if ln.startswith("checked=")]
        assert line, r.stdout + r.stderr
        kv = dict(p.split("=") for p in line[-1].split())
        return int(kv["checked"]), int(kv["bad"]), r.stdout

    return run
