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

_jobs = {"procs": [], "dir": None, "logs": []}


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: longer CPU test")
    config.addinivalue_line("markers", "oracle_job(name): compares with a long oracle computation run in the "
                                       "background (tests/oracle_jobs.py)")


def _start_oracle_jobs(names):
    """Background interpreters run the selected oracle jobs (seeded inputs only) while the tests run: one per
    group of oracle_jobs.GROUPS, each with half the host's cores."""
    import oracle_jobs as OJ

    d = tempfile.mkdtemp(prefix="cbs_oracle_jobs_")
    _jobs["dir"] = d
    env = dict(os.environ)
    env["OMP_NUM_THREADS"] = str(max(1, (os.cpu_count() or 2) // 2))
    for gi, group in enumerate(OJ.GROUPS):
        todo = [n for n in group if n in names]
        if not todo:
            continue
        log = open(os.path.join(d, f"jobs{gi}.log"), "w")
        _jobs["procs"].append(subprocess.Popen(
            [sys.executable, os.path.join(ROOT, "tests", "oracle_jobs.py"), d, *todo],
            stdout=log, stderr=subprocess.STDOUT, cwd=ROOT, env=env))
        _jobs["logs"].append(log)


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
    for p in _jobs["procs"]:
        if p.poll() is None:
            p.terminate()
            try:
                p.wait(timeout=10)
            except Exception:
                p.kill()
    for log in _jobs["logs"]:
        log.close()


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
        if all(p.poll() is not None for p in _jobs["procs"]) and not os.path.exists(path):
            text = ""
            for gi in range(len(OJ.GROUPS)):
                lp = os.path.join(_jobs["dir"], f"jobs{gi}.log")
                if os.path.exists(lp):
                    with open(lp) as f:
                        text += f.read()[-2000:]
            raise RuntimeError(f"oracle job {name} did not finish:\n{text}")
        if time.time() - t0 > 3600:
            raise TimeoutError(f"oracle job {name} still running after an hour")
        time.sleep(1.0)
    with np.load(path) as z:
        return {k: z[k] for k in z.files}
