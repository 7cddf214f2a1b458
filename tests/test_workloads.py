"""Host logic of the workload definitions (CPU): the step sizes sit inside the
stability bound the generator states, and a scaled bench catalog keeps the
recipe and the minibatch fraction of its workload."""
import importlib.util
import math
import os

import numpy as np

from paper_2508_12117_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_batched_workload_shares_one_step_size_set_by_its_densest_catalog():
    specs = synth.batch_specs(16)
    mb = specs[0].hyper.batch_n
    ratio = max(s.n_events * s.n_neighbours * 10 for s in specs) / mb
    want = synth._eps_for(0.03, 20, ratio)
    assert all(s.hyper.eps == want for s in specs)
    # every catalog's own ratio is at most the one the step size was set for
    for s in specs:
        assert s.n_events * s.n_neighbours * 10 / mb <= ratio + 1e-9


def test_full_batch_workload_step_size_counts_every_observation_of_an_event():
    s2 = synth.spec(2)
    assert s2.hyper.batch_n == 0
    assert math.isclose(s2.hyper.eps, synth._eps_for(0.03, 200, 1.0))
    # the minibatch workloads keep 20 effective observations per event
    for wid, n_obs in ((3, 50e6), (4, 200e6)):
        s = synth.spec(wid)
        assert math.isclose(s.hyper.eps, synth._eps_for(0.03, 20, n_obs / s.hyper.batch_n))


def test_bench_scaled_catalog_keeps_the_recipe_and_minibatch_fraction():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    cat, _ = bench.build_workload(4, 20000)
    full = synth.spec(4)
    assert cat.M == 20000 and cat.spec.hidden == full.hidden
    bn = cat.spec.hyper.batch_n
    assert bn % full.hyper.block_obs == 0
    frac_full = full.hyper.batch_n / 200e6
    assert abs(bn / cat.N - frac_full) <= full.hyper.block_obs / cat.N + 0.2 * frac_full
    assert np.isfinite(cat.dt).all()
