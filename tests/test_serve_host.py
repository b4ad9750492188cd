"""Host logic of the continuous-batching server (paper_2512_19847_gb300/serve.py) without a
GPU: the batch handle, the device copies and the CUDA events are replaced by fakes that
count the steps each slot is given, so that the scheduling itself is checked — every
request gets exactly its steps, slots and the HBM budget are never exceeded, admission
is in arrival order, and a request that can never fit is refused instead of waiting
forever."""
import types

import pytest
import torch

from paper_2512_19847_gb300 import serve

BASE = 1000            # bytes of the fake batch workspace
PER_CELL = 10          # fake instance bytes per cell


class FakeBatch:
    made = []

    def __init__(self, template, capacity):
        self.capacity = capacity
        self.workspace = torch.empty(BASE, dtype=torch.uint8)
        self.slots = {}                      # slot -> [params, steps done]
        self.calls = []                      # (nsteps, {slot: steps}) of every step_slots call
        self.attach_order = []
        FakeBatch.made.append(self)

    @staticmethod
    def instance_bytes(params):
        return PER_CELL * params.nx * params.ny

    def set_graph_steps(self, k):
        pass

    def set_tile(self, t):
        pass

    def attach(self, slot, params):
        assert 0 <= slot < self.capacity and slot not in self.slots
        self.slots[slot] = [params, 0]
        self.attach_order.append(params.rid)

    def set_equilibrium(self, u1, u2, p, slot=0):
        assert slot in self.slots

    def step_slots(self, nsteps, steps):
        # the C ABI's rule: every attached slot has a count in [0, nsteps]
        assert set(steps) == set(self.slots)
        assert all(0 <= c <= nsteps for c in steps.values())
        self.calls.append((nsteps, dict(steps)))
        for s, c in steps.items():
            self.slots[s][1] += c

    def get_state(self, slot):
        return torch.full((6, 2, 2), float(self.slots[slot][1]), dtype=torch.float64)

    def detach(self, slot):
        del self.slots[slot]


class FakeEvent:
    def record(self, stream=None):
        pass

    def query(self):
        return True

    def synchronize(self):
        pass


class Field:
    def to(self, *a, **k):
        return self


@pytest.fixture
def fake(monkeypatch):
    FakeBatch.made.clear()
    monkeypatch.setattr(serve.api, "Batch", FakeBatch)
    cuda = types.SimpleNamespace(Event=FakeEvent, current_stream=lambda: None, synchronize=lambda: None)
    ft = types.SimpleNamespace(empty=lambda shape, dtype=None, pin_memory=False: torch.empty(shape, dtype=dtype),
                               cuda=cuda)
    monkeypatch.setattr(serve, "torch", ft)
    return FakeBatch


def jobs_of(spec):
    """spec: (arrival, side, steps) per request."""
    out = []
    for k, (t, n, steps) in enumerate(spec):
        prm = types.SimpleNamespace(nx=n, ny=n, rid=k)
        out.append(serve.Job(k, t, prm, steps, (Field(), Field(), Field())))
    return out


def test_every_request_gets_exactly_its_steps(fake):
    spec = [(0.0, 8, 7), (0.0, 8, 25), (0.0, 4, 3), (0.001, 8, 12), (0.002, 4, 30), (0.002, 8, 1)]
    jobs = jobs_of(spec)
    srv = serve.Server(types.SimpleNamespace(), capacity=3, hbm_budget=BASE + 3 * PER_CELL * 64, chunk=10)
    st = srv.run(jobs)
    for j, (_, _, steps) in zip(jobs, spec):
        assert float(j.result[0, 0, 0]) == steps
        assert j.done >= j.admitted >= j.arrival
    assert st.cell_steps == sum(n * n * s for _, n, s in spec)
    assert st.max_resident <= 3 and st.max_bytes <= BASE + 3 * PER_CELL * 64
    b = fake.made[0]
    # each round steps by at most the chunk and no solve by more than it still needs
    assert all(n <= 10 for n, _ in b.calls)
    assert st.summary()["requests"] == len(spec)


def test_admission_is_in_arrival_order_and_within_the_budget(fake):
    # one 8x8 (640 B) fits beside the base workspace, a second does not: one at a time
    spec = [(0.0, 8, 5), (0.0, 8, 5), (0.0, 8, 5)]
    jobs = jobs_of(spec)
    srv = serve.Server(types.SimpleNamespace(), capacity=4, hbm_budget=BASE + PER_CELL * 64 + 100, chunk=4)
    st = srv.run(jobs)
    assert fake.made[0].attach_order == [0, 1, 2]
    assert st.max_resident == 1
    assert all(float(j.result[0, 0, 0]) == 5 for j in jobs)


def test_short_jobs_do_not_shrink_the_round(fake):
    # a 1-step job beside a 20-step one: rounds still advance the long one by the full chunk
    jobs = jobs_of([(0.0, 4, 1), (0.0, 4, 20)])
    srv = serve.Server(types.SimpleNamespace(), capacity=2, hbm_budget=1e9, chunk=10)
    srv.run(jobs)
    assert fake.made[0].calls == [(10, {0: 1, 1: 10}), (10, {1: 10})]


def test_a_request_that_can_never_fit_is_refused(fake):
    jobs = jobs_of([(0.0, 4, 2), (0.0, 64, 2)])          # 64^2 needs 40960 B
    srv = serve.Server(types.SimpleNamespace(), capacity=2, hbm_budget=BASE + 5000, chunk=4)
    with pytest.raises(ValueError, match="request 1"):
        srv.run(jobs)
