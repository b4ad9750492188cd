"""Host logic of the tile autotuner (paper_2512_19847_gb300/autotune.py) without a GPU: a
fake handle whose step time depends on the tile shape, and fake CUDA events on a fake
clock.  Checked: the fastest admissible tile is chosen and set, tiles larger than the
smallest attached grid are never tried, the solves' state (FP64 moments, FP32 populations,
the carried theta plane) is put back exactly, and the cache answers a second call without
stepping."""
import types

import pytest
import torch

from paper_2512_19847_gb300 import api, autotune

COST_MS = {0: 3.0, 1: 2.5, 2: 1.5, 3: 4.0, 4: 2.0, 5: 1.0}   # ms per step of each tile shape


class Clock:
    t = 0.0


class FakeEvent:
    def __init__(self, enable_timing=False):
        self.at = None

    def record(self, stream=None):
        self.at = Clock.t

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return other.at - self.at


class FakeHandle:
    def __init__(self, grids):
        self._params = {}
        self.state = {}
        self.theta = {}
        for slot, (nx, ny, prec) in enumerate(grids):
            self._params[slot] = types.SimpleNamespace(nx=nx, ny=ny, precision=prec, space_scheme=2, s=3)
            g = torch.Generator().manual_seed(slot)
            self.state[slot] = torch.randn((6, ny, nx), generator=g, dtype=torch.float64)
            self.theta[slot] = self.state[slot][2].clone()
        self.tile = None
        self.tried = []
        self.steps = 0

    def set_tile(self, t):
        self.tile = t
        self.tried.append(t)

    def step(self, n):
        self.steps += n
        Clock.t += n * COST_MS[self.tile]
        for s in self.state:                       # stepping changes every solve
            self.state[s] = self.state[s] * 1.01 + 0.5
            self.theta[s] = self.theta[s] - 1.0

    def get_state(self, slot):
        X = self.state[slot].clone()
        X[2] = self.theta[slot]
        return X

    def set_state(self, X, slot):
        self.state[slot] = X.clone()
        self.theta[slot] = X[2].clone()

    def get_populations(self, slot, dtype):
        return self.state[slot].to(dtype)

    def set_populations(self, F, slot):
        self.state[slot] = F.to(torch.float64)

    def set_theta(self, th, slot):
        self.theta[slot] = th.clone()


@pytest.fixture
def fake(monkeypatch):
    cuda = types.SimpleNamespace(Event=FakeEvent, current_stream=lambda: None, synchronize=lambda: None,
                                 get_device_name=lambda: "fake GPU")
    monkeypatch.setattr(autotune, "torch", types.SimpleNamespace(float32=torch.float32, cuda=cuda))


def snapshot(h):
    return {s: (h.state[s].clone(), h.theta[s].clone()) for s in h.state}


def test_fastest_tile_is_chosen_and_state_restored(fake, tmp_path):
    # FP32 populations round-trip through float32: start from values float32 holds exactly
    h = FakeHandle([(64, 64, api.FP64), (48, 32, api.FP32_DEV), (64, 48, api.FP32_DEV_TH)])
    for s in (1, 2):
        h.state[s] = h.state[s].to(torch.float32).to(torch.float64)
    before = snapshot(h)
    r = autotune.tune(h, steps=2, path=str(tmp_path / "c.json"))
    assert r["tile"] == 5 and h.tile == 5 and not r["cached"]
    assert r["ms_per_step"]["5"] == pytest.approx(1.0) and r["ms_per_step"]["3"] == pytest.approx(4.0)
    after = snapshot(h)
    for s in before:
        assert torch.equal(before[s][0], after[s][0])
        if h._params[s].precision != api.FP32_DEV:   # FP32_DEV carries no theta plane
            assert torch.equal(before[s][1], after[s][1])


def test_tiles_larger_than_a_grid_are_not_tried(fake):
    h = FakeHandle([(16, 8, api.FP64), (256, 256, api.FP64)])
    assert autotune.candidates(h) == [2, 3]                  # 16x8 and 8x8 only
    r = autotune.tune(h, steps=1, path=None)
    assert r["tile"] == 2 and set(h.tried) == {2, 3}


def test_cache_answers_without_stepping(fake, tmp_path):
    path = str(tmp_path / "c.json")
    h = FakeHandle([(64, 64, api.FP64)])
    first = autotune.tune(h, steps=1, path=path)
    h2 = FakeHandle([(64, 64, api.FP64)])
    second = autotune.tune(h2, steps=1, path=path)
    assert second["cached"] and second["tile"] == first["tile"] == h2.tile and h2.steps == 0
    # another multiset of grids is another key
    h3 = FakeHandle([(64, 64, api.FP64), (64, 64, api.FP64)])
    assert autotune.signature(h3) != autotune.signature(h)
    assert not autotune.tune(h3, steps=1, path=path)["cached"]


def test_signature_ignores_slot_order(fake):
    a = FakeHandle([(64, 32, api.FP64), (128, 128, api.FP64)])
    b = FakeHandle([(128, 128, api.FP64), (64, 32, api.FP64)])
    assert autotune.signature(a) == autotune.signature(b)
