"""Host-side logic of bench.py that needs no GPU: workload table, the replica
(N > 1) timing reduction over a gloo process group, the clock summary."""
import os
import socket
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_workloads():
    w = bench.workload("dvr1024")
    assert w["dims"] == (1024, 1024, 1024) and w["views"] == 32 and (w["W"], w["H"]) == (1920, 1080)
    assert w["step"] == 0.5 and w["nbins"] == 4096 and w["term"] == 0.99
    assert bench.workload("small128")["dims"] == (128, 128, 128)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_replica_max_over_ranks_gloo(tmp_path):
    script = tmp_path / "w.py"
    script.write_text(textwrap.dedent(f"""
        import os, sys
        sys.path.insert(0, {ROOT!r})
        import torch.distributed as dist
        import bench
        dist.init_process_group("gloo")
        r = dist.get_rank()
        m = bench.barrier_max(1.0 + r * 2.5, dist.get_world_size())
        bench.barrier(dist.get_world_size())
        print("RESULT", r, m)
        dist.destroy_process_group()
    """))
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env, stdout=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120)[0] for p in procs]
    assert all(p.returncode == 0 for p in procs)
    vals = [float(o.split("RESULT")[1].split()[1]) for o in outs]
    assert vals == [3.5, 3.5]


def test_clock_summary_parsing():
    c = bench.Clocks(0)
    c.proc = None
    assert c.stop()["sm_mhz"] is None
