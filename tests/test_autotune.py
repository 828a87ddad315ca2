"""Autotuner selection rule (CPU) and a tiny end-to-end tuning run (GPU)."""
import pytest

from paper_2606_26010_gb300.autotune import Trial, select


def T(v, tpp, lf, ms, err):
    return Trial(v, tpp, lf, ms, 1.0 / ms, err, 0.0, 0)


def test_select_fastest_within_accuracy_margin():
    trials = [T(0.25, 1, 0.5, 9.0, 0.010), T(0.5, 4, 0.5, 5.0, 0.012), T(1.0, 4, 0.5, 2.0, 0.20),
              T(0.5, 8, 0.3, 4.0, 0.013)]
    best = select(trials, err_margin=1.5, err_floor_m=0.005)
    assert (best.voxel_size, best.threads_per_point, best.load_factor) == (0.5, 8, 0.3)
    # a generous floor admits the fast but inaccurate candidate
    assert select(trials, err_margin=1.5, err_floor_m=0.5).voxel_size == 1.0


@pytest.mark.gpu
def test_autotune_runs_on_small_problems():
    import torch
    import synth
    from paper_2606_26010_gb300 import autotune, build
    build.build()
    seq, specs = synth.batched_problems(3, 3, scan_range=(5e3, 2e4), map_range=(5e4, 1e5), max_prior=6)
    cache = {}

    def scan_dev(i):
        if i not in cache:
            cache[i] = torch.from_numpy(seq.scan(i)).cuda()
        return cache[i]

    qs = [torch.from_numpy(sp.query).cuda() for sp in specs]
    grid = {"voxel_size": (0.5, 1.0), "threads_per_point": (1, 4), "load_factor": (0.5,)}
    best, trials = autotune.autotune(scan_dev, seq.pose, specs, qs, grid=grid, reps=2, max_iters=10, tau=2.0,
                                     kappa=0.25)
    assert len(trials) == 4 and best in trials
    assert best.median_trans_err_m < 0.5
