"""The multi-rank plumbing of bench.py on CPU: world_size 2 over gloo (127.0.0.1).

The path shards as replicas (every rank unfolds its own copy of the workload, no data-path
collective); what crosses ranks is only the barrier and the max over ranks of the timed
region, which this test exercises with the same helpers bench.py uses."""
import os
import socket
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_max_and_barrier(tmp_path):
    script = tmp_path / "ranks.py"
    script.write_text(textwrap.dedent(f"""
        import os, sys
        sys.path.insert(0, {ROOT!r})
        import bench
        world, rank, local = bench.dist_setup(False)
        assert world == 2
        bench.barrier(world)
        m = bench.allmax(world, float(10 + rank))
        assert m == 11.0, m
        print("rank", rank, "ok", m)
    """))
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(r), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.STDOUT, text=True))
    outs = [p.communicate(timeout=120)[0] for p in procs]
    for p, o in zip(procs, outs):
        assert p.returncode == 0, o
    assert "rank 0 ok 11.0" in outs[0] and "rank 1 ok 11.0" in outs[1]


def test_reference_arm_rank_nonzero_exits_quietly():
    port = _free_port()
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(port))
    # rank 1 of the reference arm returns before any rendezvous work is needed beyond init;
    # run both ranks so the gloo group forms
    env0 = dict(env, RANK="0", LOCAL_RANK="0")
    p0 = subprocess.Popen([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "3"], env=env0, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    p1 = subprocess.Popen([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "3"], env=env, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    o1 = p1.communicate(timeout=300)[0]
    o0 = p0.communicate(timeout=300)[0]
    assert p0.returncode == 0 and p1.returncode == 0, (o0, o1)
    assert '"impl": "reference"' in o0 and '"impl"' not in o1
