"""The replica path of bench.py on CPU with two gloo ranks: the timing
reductions (max over ranks of the time, sum over ranks of the work) and the
reference arm under torchrun (rank 0 alone runs and prints one line)."""
import json
import os
import socket
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def torchrun(args, timeout):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port())] + args
    return subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=timeout)


def test_reductions_over_two_gloo_ranks(tmp_path):
    script = tmp_path / "ranks.py"
    script.write_text(textwrap.dedent(f"""
        import sys
        sys.path.insert(0, {ROOT!r})
        import bench
        world, rank, local, pg = bench.dist_setup(2)
        assert world == 2 and pg is not None
        bench.barrier(pg)
        ms = 10.0 + 5.0 * rank          # rank 1 is the slower one
        work = 1000.0 * (rank + 1)
        assert bench.allmax(pg, ms) == 15.0
        assert bench.allsum(pg, work) == 3000.0
        # the aggregate rate: all ranks' work over the slowest rank's time
        # (one file per rank: the ranks' stdout lines may interleave)
        rate = bench.allsum(pg, work) / (bench.allmax(pg, ms) / 1e3)
        open({str(tmp_path)!r} + "/rate%d" % rank, "w").write(repr(rate))
        pg.destroy_process_group()
    """))
    r = torchrun([str(script)], timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    rates = [float((tmp_path / ("rate%d" % k)).read_text()) for k in range(2)]
    assert rates == [200000.0, 200000.0]


def test_reference_arm_under_torchrun_prints_one_line():
    r = torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                  "--warmup", "3"], timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["value"] > 0 and out["steps"] == 1
