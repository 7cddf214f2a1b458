"""Host logic of the launch-shape autotuner, on the CPU with a stand-in context:
every candidate is timed, the fastest is kept and applied, the chain state is
restored afterwards, and a second call with the cache takes the stored choice
without stepping."""
import time

from paper_2508_12117_gb300 import autotune
from paper_2508_12117_gb300.binding import BF16, FP32


class FakeContext:
    """Duck-types the calls the autotuner makes; a step sleeps for a time that
    depends on the current knobs, with (2, 1, f, 1, 2, 2) the fastest."""

    def __init__(self):
        self.knobs = None
        self.steps = 0
        self.state = ("theta0", 7)
        self.restored = None
        self.applied = []

    def spider_info(self):
        return {"n_sub": 4, "events": 1000, "obs": 50000, "blocks_per_step": 8}

    def spider_set_tuning(self, knobs):
        self.knobs = tuple(knobs)
        self.applied.append(self.knobs)

    def spider_sgld_step(self, eps, seed):
        w, c, f, _, q, t = self.knobs
        time.sleep(0.002 * (abs(w - 2) + abs(c - 1) + abs(q - 2) + abs(t - 2)) + 0.0005)
        self.steps += 1

    def spider_sync(self):
        pass

    def spider_get_state(self):
        return self.state

    def spider_set_state(self, theta, step):
        self.restored = (theta, step)


def test_candidates_cover_the_knobs():
    assert len(autotune.candidates(FP32)) == 108         # 3 warp x 2 CTA x 2 FP32-MLP x 3 clean x 3 CTA sizes
    assert len(autotune.candidates(BF16)) == 54
    assert all(k[2] == 2 and k[3] == 1 for k in autotune.candidates(BF16))


def test_autotune_picks_fastest_restores_state_and_caches(tmp_path):
    path = str(tmp_path / "tune.json")
    ctx = FakeContext()
    knobs, timings = autotune.autotune(ctx, 1e-4, BF16, 128, steps=2, path=path, use_cache=True)
    assert knobs == (2, 1, 2, 1, 2, 2)
    assert ctx.knobs == (2, 1, 2, 1, 2, 2)                # the choice is left applied
    assert ctx.restored == ctx.state                      # tuning does not advance the sampler
    assert len(timings) == len(autotune.candidates(BF16))
    assert ctx.steps == 3 * len(timings)                  # one capture step + 2 timed per candidate

    again = FakeContext()
    k2, t2 = autotune.autotune(again, 1e-4, BF16, 128, path=path, use_cache=True)
    assert k2 == (2, 1, 2, 1, 2, 2) and t2 == {} and again.steps == 0
    assert again.applied == [(2, 1, 2, 1, 2, 2)]


def test_signature_separates_workloads():
    a = FakeContext()
    b = FakeContext()
    b.spider_info = lambda: {"n_sub": 4, "events": 2000, "obs": 50000, "blocks_per_step": 8}
    assert autotune.signature(a, BF16, 128) != autotune.signature(b, BF16, 128)
    assert autotune.signature(a, BF16, 128) != autotune.signature(a, FP32, 128)
