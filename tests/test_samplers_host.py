"""Host-side sampler logic that needs no GPU: the per-step metric records
(JSONL) built from the reweight scalars."""
import json

import numpy as np

from paper_0905_2441_gb300 import samplers


def test_step_records_and_jsonl(tmp_path):
    M = 1000
    betas = np.array([0.0, 0.1, 0.4, 1.0])
    hist = np.array([[0, 0, 0, 0], [-1.5, 900.0, 0, 0], [-2.0, 400.0, 0, 0], [-0.5, 950.0, 0, 0]])
    flags = np.array([0, 0, 1, 0], np.int32)
    accepts = np.array([0, 500, 700, 300], np.int32)
    rec = samplers.step_records(hist, betas, M, flags, accepts, n_moves=2)
    assert [r["t"] for r in rec] == [1, 2, 3]
    assert [r["resampled"] for r in rec] == [False, True, False]
    np.testing.assert_allclose([r["log_z"] for r in rec], [-1.5, -3.5, -4.0])
    np.testing.assert_allclose([r["accept_rate"] for r in rec], [0.25, 0.35, 0.15])
    np.testing.assert_allclose([r["ess_frac"] for r in rec], [0.9, 0.4, 0.95])
    p = tmp_path / "run.jsonl"
    samplers.write_jsonl(rec, p)
    back = [json.loads(line) for line in p.read_text().splitlines()]
    assert back == rec
    # without flags / acceptance counts the records hold the weights only
    assert "resampled" not in samplers.step_records(hist, betas, M)[0]
