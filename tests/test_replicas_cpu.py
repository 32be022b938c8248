"""The replicas-only multi-GPU path of bench.py, on CPU with gloo at world size 2 (the path has no
exchange step, so a run on N GPUs is N independent replicas):

- the job's step time is the slowest rank's: every rank gets the maximum over ranks;
- every rank builds its own workload (its own seeded scene and view);
- the reference arm runs on rank 0 only, where it prints one line with the contract keys; other
  ranks exit 0 without work or output.
"""
import json
import os
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_RANK_SCRIPT = textwrap.dedent("""
    import json, sys
    import numpy as np
    sys.path.insert(0, {root!r})
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo")
    r = dist.get_rank()
    t = bench.max_over_ranks(10.0 + 3.0 * r, "cpu")
    scene, cams = bench.make_workload(r, n=2000, width=64, height=48)
    # one file per rank: the ranks share one stdout, where their lines can interleave
    with open(f"rank{{r}}.json", "w") as f:
        json.dump({{"rank": r, "t": t, "mean0": [float(x) for x in scene.means[0]],
                   "pose": [float(x) for x in np.asarray(cams[0].world_to_cam).reshape(-1)]}}, f)
    dist.destroy_process_group()
""")


def test_two_gloo_ranks_share_the_max_and_build_their_own_workloads(tmp_path):
    script = tmp_path / "rank.py"
    script.write_text(_RANK_SCRIPT.format(root=ROOT))
    # --standalone picks a free rendezvous port itself
    cmd = [sys.executable, "-m", "torch.distributed.run", "--standalone", "--local-addr=127.0.0.1",
           "--nnodes=1", "--nproc-per-node=2", str(script)]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, env=env, cwd=str(tmp_path))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.load(open(tmp_path / f"rank{k}.json")) for k in (0, 1)]
    by = {d["rank"]: d for d in lines}
    assert sorted(by) == [0, 1]
    assert by[0]["t"] == by[1]["t"] == 13.0
    # weak scaling: each rank has its own scene and view
    assert by[0]["mean0"] != by[1]["mean0"]
    assert by[0]["pose"] != by[1]["pose"]


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1"],
                       capture_output=True, text=True, timeout=300, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_single_rank_max_is_the_value_itself():
    import bench
    assert bench.max_over_ranks(7.5, "cpu") == 7.5


def test_reference_arm_prints_one_line_with_the_contract_keys():
    """Rank 0 of the reference arm (the FP64 oracle on a small pixel sample per step) prints one
    JSON line with the render metric, its own cpu_baseline and an e2e entry without copies."""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", CUDA_VISIBLE_DEVICES="", SOF_REF_PIXELS="4")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 3 and d["higher_is_better"] is False
    import bench
    assert d["metric"] == bench.METRIC and d["unit"] == "ms" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and "4 random pixels" in d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
