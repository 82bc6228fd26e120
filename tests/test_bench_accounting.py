"""bench.py's algorithmic byte count (A_min and the looser A_pair) on small batches, CPU only."""
import numpy as np

import bench
import oracle
import synth


def _acc(c, batch, p=4, q=5):
    return bench.oracle_accounting([c], [(0, p, q, batch.probe_ids, batch.cand_offsets, batch.cand_ids)])[0]


def test_a_min_formula_and_a_pair_bound():
    c = synth.collection(synth.tiny_self_join(seed=1001, n=200))
    b = synth.all_pairs_batch(c.n)
    a = _acc(c, b)
    tr, cr, cs = oracle.verify_batch(c.offsets, c.tokens, c.offsets, c.tokens, True, 4, 5, b.probe_ids,
                                     b.cand_offsets, b.cand_ids, consumed=True)
    n_pr, n_ci = len(b.probe_ids), len(b.cand_ids)
    counts = np.diff(b.cand_offsets.astype(np.int64))
    starts = b.cand_offsets[:-1].astype(np.int64)
    # the probe's tokens once per probe: the deepest stop point among its candidates
    max_r = sum(int(cr[s:s + k].max()) for s, k in zip(starts, counts) if k)
    want = 12 * n_pr + 4 * n_ci + 8 * (n_pr + n_ci) + 4 * max_r + 4 * int(cs.sum()) + 12 * len(tr) + 8
    assert a["bytes"] == want
    assert a["hbm_bytes"] == 12 * n_pr + 4 * n_ci + 12 * len(tr) + 8
    assert a["pair_bytes"] - a["bytes"] == 4 * (int(cr.sum()) - max_r) >= 0
    assert a["survivors"] == len(tr) and a["pairs"] == n_ci


def test_a_pair_equals_a_min_with_one_candidate_per_probe():
    c = synth.collection(synth.tiny_self_join(seed=7, n=100))
    probes = np.arange(0, 50, dtype=np.uint32)
    cands = np.arange(50, 100, dtype=np.uint32)
    b = synth.Batch(probes, np.arange(51, dtype=np.uint64), cands)
    a = _acc(c, b, 3, 5)
    assert a["pair_bytes"] == a["bytes"]


def test_stride_sample_takes_whole_probes_at_a_uniform_stride():
    """The CPU baseline's sample: every k-th probe of each batch with all of its candidates (not a
    prefix of the feeder's size-ordered probes), about the asked number of candidates."""
    batches = []
    for seed, probes, per in ((3, 400, 60), (4, 250, 30)):
        b = synth.random_batch(seed, 500, 500, probes, per)
        batches.append((0, 3, 5, b.probe_ids, b.cand_offsets, b.cand_ids))
    total = sum(len(b[5]) for b in batches)
    sample, k = bench.stride_sample(batches, total // 7)
    assert k == -(-total // (total // 7))
    for (_, _, _, pr, co, ci), (_, _, _, spr, sco, sci) in zip(batches, sample):
        pick = np.arange(0, len(pr), k)
        assert np.array_equal(spr, pr[pick])
        co64 = co.astype(np.int64)
        want = np.concatenate([ci[co64[a]:co64[a + 1]] for a in pick])
        assert np.array_equal(sci, want)
        assert int(sco[0]) == 0 and int(sco[-1]) == len(sci) and len(sco) == len(spr) + 1
    whole, k1 = bench.stride_sample(batches, total)
    assert k1 == 1 and whole is batches


def test_both_arms_report_the_same_config():
    """The GPU arm and the reference arm build their `config` with the same function from the same
    workload and candidates, so the two lines can be compared key by key."""
    import types
    args = types.SimpleNamespace(sim="jaccard", ppjoin=False, workload="short_sets", l2_flush_mb=512)
    cfg = {"workload": "short_sets", "n_sets": 10}
    c = synth.collection(synth.tiny_self_join(seed=1001, n=50))
    b = synth.random_batch(1, 50, 50, 20, 5)
    batches = [(0, 3, 5, b.probe_ids, b.cand_offsets, b.cand_ids)]
    c1, c2 = bench.common_config(cfg, [c], batches, args), bench.common_config(dict(cfg), [c], batches, args)
    assert c1 == c2 and c1["pairs_per_step"] == len(b.cand_ids) and c1["instances_per_launch"] == 1
    nbytes = 4 * len(c.tokens) + 8 * c.n + 4 * len(b.probe_ids) + 8 * len(b.cand_offsets) + 4 * len(b.cand_ids)
    assert bench.input_bytes_of([c], batches) == nbytes
    assert "within the 129 MB L2" in c1["l2_between_steps"] and "512 MiB" in c1["l2_between_steps"]


def _bench_reference(env_extra):
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "tiny", "--steps", "2",
                        "--warmup", "3"], cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    return [json.loads(ln) for ln in lines]


def test_reference_arm_prints_one_line_of_the_contract():
    """`bench.py --impl reference` runs the oracle on the CPU (no GPU needed) and prints one JSON
    line with the GPU arm's metric, unit and config, its own cpu_baseline and a copy-free e2e."""
    (line,) = _bench_reference({"RANK": "0", "WORLD_SIZE": "1"})
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["steps"] == 2 and line["warmup"] == 3 and line["higher_is_better"]
    assert line["config"]["workload"] == "tiny" and line["config"]["pairs_per_step"] == 499_500
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"]
    assert "3 untimed warm-up steps" in cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_runs_on_rank_0_only():
    """Under torchrun the reference arm's ranks other than 0 exit 0 without work or output."""
    assert _bench_reference({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []


def test_every_profile_command_runs_committed_files_with_flags_bench_accepts():
    """Each summary under profiles/ gives the command that made it: an ncu run with
    --clock-control none of `python bench.py ...`, whose arguments the current bench.py parser
    still accepts (workload, granularity setting, flags)."""
    import glob
    import os
    import re
    import shlex
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    files = sorted(glob.glob(os.path.join(root, "profiles", "*.md")))
    assert files
    for f in files:
        text = open(f).read()
        blocks = re.findall(r"```\n(.*?)```", text, flags=re.S)
        cmds = [b.replace("\\\n", " ") for b in blocks if "bench.py" in b]
        assert cmds, f"{f} gives no command"
        for cmd in cmds:
            cmd = " ".join(cmd.split())
            assert cmd.startswith("ncu ") and "--clock-control none" in cmd, f
            tail = cmd.split("python bench.py", 1)[1]
            args = bench.build_parser().parse_args(shlex.split(tail))
            assert args.warmup >= 3, f
            if args.granularity:
                bench.parse_granularity(args.granularity)


def test_parse_granularity():
    assert bench.parse_granularity("512,2048,2048,256") == (512, 2048, 2048, 256, 0, 0)
    assert bench.parse_granularity("4096,1,4096,65664,16,256") == (4096, 1, 4096, 65664, 16, 256)
    for bad in ("1,2,3", "1,2,3,4,5,6,7", "1,-2,3,4"):
        try:
            bench.parse_granularity(bad)
        except ValueError:
            continue
        raise AssertionError(bad)
