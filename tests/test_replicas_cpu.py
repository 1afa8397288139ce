"""The multi-GPU form is replicas only (plans are independent): each rank
plans its own disjoint slice of the batch, with no collective in the data
path; the benchmark takes the max of the ranks' times.  These host pieces run
here as two gloo ranks on the CPU."""
import json
import os
import socket
import subprocess
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_replicas_take_disjoint_plans_and_the_slowest_time():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(r),
                   LOCAL_RANK=str(r), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, os.path.join(HERE, "_replica_rank.py")], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=300) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e[-2000:]
    res = json.loads(outs[0][0].strip().splitlines()[-1])
    assert res["t"] == 2.5                                   # max over ranks
    g0, g1 = np.array(res["goals"][0]), np.array(res["goals"][1])
    assert g0.shape == g1.shape == (3, 2)
    assert not np.any(np.all(np.isclose(g0[:, None, :], g1[None, :, :]), axis=-1))   # disjoint plans
