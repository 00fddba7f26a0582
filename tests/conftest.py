import os
import subprocess
import sys
import tempfile
import time

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for _p in (ROOT, HERE):
    if _p not in sys.path:
        sys.path.insert(0, _p)

_jobs = {"proc": None, "dir": None, "log": None}


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: longer CPU test")
    config.addinivalue_line("markers", "oracle_job(name): compares with a long oracle computation run in the "
                                       "background (tests/oracle_jobs.py)")


def _start_oracle_jobs(names):
    """One background interpreter runs the selected oracle jobs (seeded inputs only) while the tests run."""
    import oracle_jobs as OJ

    order = [n for n in OJ.ORDER if n in names]
    d = tempfile.mkdtemp(prefix="cbs_oracle_jobs_")
    log = open(os.path.join(d, "jobs.log"), "w")
    _jobs["proc"] = subprocess.Popen([sys.executable, os.path.join(ROOT, "tests", "oracle_jobs.py"), d, *order],
                                     stdout=log, stderr=subprocess.STDOUT, cwd=ROOT)
    _jobs["dir"], _jobs["log"] = d, log


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:
        have_gpu = False
    if not have_gpu:
        skip = pytest.mark.skip(reason="no CUDA device")
        for it in items:
            if "gpu" in it.keywords:
                it.add_marker(skip)
        return
    names = {m.args[0] for it in items for m in it.iter_markers("oracle_job")}
    if names:
        _start_oracle_jobs(names)


def pytest_unconfigure(config):
    p = _jobs["proc"]
    if p is not None and p.poll() is None:
        p.terminate()
        try:
            p.wait(timeout=10)
        except Exception:
            p.kill()
    if _jobs["log"] is not None:
        _jobs["log"].close()


@pytest.fixture
def oracle_job(request):
    """Load the result of the background oracle job named by the test's oracle_job marker (waits for it)."""
    import numpy as np

    import oracle_jobs as OJ

    name = request.node.get_closest_marker("oracle_job").args[0]
    assert _jobs["dir"] is not None, "oracle jobs were not started"
    path = OJ.job_path(_jobs["dir"], name)
    t0 = time.time()
    while not os.path.exists(path):
        p = _jobs["proc"]
        if p.poll() is not None and not os.path.exists(path):
            with open(os.path.join(_jobs["dir"], "jobs.log")) as f:
                raise RuntimeError(f"oracle job {name} did not finish (exit {p.returncode}):\n{f.read()[-4000:]}")
        if time.time() - t0 > 3600:
            raise TimeoutError(f"oracle job {name} still running after an hour")
        time.sleep(1.0)
    with np.load(path) as z:
        return {k: z[k] for k in z.files}
