"""The bench's CPU legs on a small pangenome: the oracle samples it prints
beside the GPU figures run, and say what they timed.  CPU only."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
import oracle  # noqa: E402
import synth  # noqa: E402


def test_diversity_cpu_sample_runs_the_oracle():
    S = synth.pangenome(seed=5, founder_len=30_000, n_hap=5, batch=5)
    r = bench.diversity_cpu_sample(S, window=3_000, k=51, nq=20)
    assert r["kind"] == "oracle" and r["unit"] == "queries/s" and r["cores"] == 1
    assert r["value"] > 0 and "20 sliding 51-mers" in r["sample"]
    # the sample's index is the oracle's BWT of the windows, both strands
    wins = [S.seq[o:o + 3_000] for o in S.offsets[:-1]]
    n = 2 * (sum(len(w) for w in wins) + len(wins))
    assert f"({n} symbols)" in r["sample"]
    assert len(oracle.bwt(oracle.concat(np.concatenate(wins), np.array([len(w) for w in wins]), True))) == n
