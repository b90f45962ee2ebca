"""The learned batch-split cost model: its GPU training kernels against the
CPU reference (gradients), that training fits, and what the trained model
gains over choosing the default split, on batches it was not trained on."""
from __future__ import annotations

import numpy as np
import pytest

import cg_synth as S
from oracle import mlp as M
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cg():
    import torch
    assert torch.cuda.is_available()
    import paper_1310_0901_gb300 as m
    return m


@pytest.mark.parametrize("hidden,n", [(32, 7), (32, 300), (64, 1000)])
def test_gpu_gradients_match_cpu_reference(cg, hidden, n):
    rng = np.random.default_rng(hidden + n)
    x = (rng.normal(size=(n, M.D)) * 2 + 1).astype(np.float32)
    t = rng.normal(size=n).astype(np.float32)
    w = np.zeros(cg.mlp_nweights(hidden), np.float32)
    w[:M.D] = x.mean(axis=0)
    w[M.D:2 * M.D] = x.std(axis=0) + 0.1
    w[2 * M.D:] = (rng.normal(size=w.size - 2 * M.D) * 0.3).astype(np.float32)
    g_gpu, l_gpu = cg.mlp_grad(x, t, w, hidden)
    g_cpu, l_cpu = M.grad(x.astype(np.float64), t.astype(np.float64), w.astype(np.float64),
                          hidden)
    assert abs(l_gpu - l_cpu) <= 1e-4 * max(1.0, abs(l_cpu))
    scale = np.abs(g_cpu).max()
    assert np.max(np.abs(g_gpu - g_cpu)) <= 2e-4 * scale, np.max(np.abs(g_gpu - g_cpu)) / scale


def test_fit_reduces_loss(cg):
    rng = np.random.default_rng(5)
    x = rng.normal(size=(400, M.D)).astype(np.float32)
    t = (np.sin(x[:, 0]) + 0.5 * x[:, 1] ** 2 - x[:, 13]).astype(np.float32)
    w, losses = cg.mlp_fit(x, t, 32, 1500, 3e-3, 0)
    assert losses[-1] < 0.1 * losses[0]
    assert abs(M.loss(x, t, w, 32) - losses[-1]) < 0.05 * losses[0]


def test_learned_split_gains_over_default(cg):
    """On batch shapes the model was not trained on, drawn from four
    families where the best split differs, the model's choice must beat the
    library's fixed fallback (64 KiB, what a batch of a new shape gets with
    no tuned entry, no online trials and no model) by more than the noise of
    repeated dry runs, and come close to the per-batch grid-search best."""
    from paper_1310_0901_gb300 import costmodel as CM
    rng = S.rng_for(31)
    table = S.alloc_table(rng, 20000, 256, 1 << 20, log_sizes=True)
    img = S.host_image_runs(rng, 256 << 20, 1e-4, 8.0, 0.5, 1e-5)
    ctx, _, _ = U.make_pair(img, table)
    train_b = [S.tuning_batch_mixed(rng, table, img.n) for _ in range(128)]
    held_rng = S.rng_for(97)  # held-out shapes: another stream
    held_b = [S.tuning_batch_mixed(held_rng, table, img.n) for _ in range(32)]
    train = CM.measure(ctx, train_b, repeats=2)
    held = CM.measure(ctx, held_b, repeats=2)
    # noise: the fallback's total time over the held-out batches, measured again
    again = sum(ctx.tune_batch(b, [64], 2, remember=False)[1][64] for b in held_b)
    first = sum(m["ms"][64] for m in held)
    noise = abs(again - first) / first
    w, losses = CM.fit(train, hidden=32, epochs=4000)
    assert losses[-1] < losses[0]
    ctx.set_cost_model(w, 32)
    t_default = t_model = t_best = 0.0
    t_const = {k: 0.0 for k in cg.CANDIDATES_KIB}
    for b, m in zip(held_b, held):
        kib, source = ctx.choose_segment(b)
        assert source == 2
        preds = {k: CM.predict(w, m["features"], k, 32) for k in cg.CANDIDATES_KIB}
        assert kib == min(preds, key=preds.get)
        t_default += m["ms"][64]
        t_model += m["ms"][kib]
        t_best += min(m["ms"].values())
        for k in t_const:
            t_const[k] += m["ms"][k]
    best_const = min(t_const, key=t_const.get)
    margin = max(0.05, 3 * noise)
    print(f"held-out level time over {len(held_b)} batches: fallback 64 KiB {t_default:.2f} ms, "
          f"learned {t_model:.2f} ms (gain {t_default / t_model:.3f}x), grid-search best "
          f"{t_best:.2f} ms, best fixed size {best_const} KiB {t_const[best_const]:.2f} ms; "
          f"dry-run noise {noise:.3f}")
    assert t_model < t_default * (1 - margin)
    assert t_model <= t_best * 1.10
    # a tuned entry for a batch takes precedence over the model
    best, _ = ctx.tune_batch(held_b[1], repeats=1)
    assert ctx.choose_segment(held_b[1]) == (best, 1)


def test_online_autotune_tries_then_keeps_fastest(cg):
    """With batch_autotune on, batches of one shape try the candidates in
    turn (real runs) and then keep the fastest; every batch's reports stay
    equal to the oracle's whatever the split."""
    import oracle as O
    w = S.small(5)
    ctx, orc, (a, v) = U.make_pair(w.image, w.table, batch_autotune=1)
    seen = []
    for rep in range(7):
        kib, source = ctx.choose_segment(w.reqs)
        seen.append((kib, source))
        st, reps, recs, total, _ = ctx.check_batch(w.reqs)
        assert st == 0
        st_o, oreps, _ = orc.check_batch(w.reqs)
        for i, (g, o) in enumerate(zip(U.reports_from_array(reps), oreps)):
            U.assert_same_report(g, o, f"batch {rep} request {i}")
        assert U.reports_from_array(recs) == O.emit_records(oreps, w.reqs)
    trials = [k for k, s in seen if s == 4]
    assert trials == [16, 32, 64, 128, 256]
    assert seen[5][1] == 1 and seen[6] == seen[5] and seen[5][0] in trials
    U.assert_same_state(ctx, orc, v, w.table)


def test_tuned_entries_survive_save_and_load(cg, tmp_path):
    """Tuned split entries written to JSON and loaded into a fresh context
    choose the same segment size (source 1) for the same batch."""
    import json
    w = S.small(7)
    ctx, _, _ = U.make_pair(w.image, w.table)
    best, _ = ctx.tune_batch(w.reqs, repeats=1)
    assert ctx.choose_segment(w.reqs) == (best, 1)
    path = str(tmp_path / "tuned.json")
    assert ctx.save_tuning(path) == 1
    d = json.load(open(path))
    assert d["nfeat"] == cg.NFEAT and d["segment_kib"] == [best]
    ctx2, _, _ = U.make_pair(w.image, w.table)
    assert ctx2.choose_segment(w.reqs)[1] != 1
    assert ctx2.load_tuning(path) == 1
    assert ctx2.choose_segment(w.reqs) == (best, 1)
    d["segment_kib"] = [0]
    json.dump(d, open(path, "w"))
    with pytest.raises(cg.CgError):
        cg.Context().load_tuning(path)
