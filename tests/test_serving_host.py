"""Host logic of the serving layer, without a GPU: the admission controller
(FIFO by device-memory budget, head of line waits) against an independent
model of the policy, and the admission cost of a scene."""

import numpy as np
import pytest

from paper_1410_0925_gb300 import Admission, TsdfError, scene_device_bytes
from paper_1410_0925_gb300.tsdf import STORAGE_F16, STORAGE_F32, STORAGE_I16


def test_fifo_budget_and_slots():
    a = Admission(budget_bytes=100, max_active=3)
    for sid, b in [(1, 40), (2, 50), (3, 20), (4, 5)]:
        a.enqueue(sid, b)
    assert a.admit() == [1, 2]               # 3 would exceed 100 bytes
    assert a.stats() == {"active_bytes": 90, "active": 2, "queued": 2}
    assert a.admit() == []                   # head of line (3, 20) waits; 4 does not overtake
    a.release(1)
    assert a.admit() == [3, 4]               # 50 + 20 + 5 = 75
    a.enqueue(5, 1)
    assert a.admit() == []                   # three slots taken
    a.release(2)
    assert a.admit(capacity=0) == []
    assert a.admit() == [5]
    assert a.stats() == {"active_bytes": 26, "active": 3, "queued": 0}


def test_invalid_operations():
    a = Admission(budget_bytes=100, max_active=2)
    with pytest.raises(TsdfError):
        a.enqueue(1, 101)                    # can never fit
    with pytest.raises(TsdfError):
        a.enqueue(1, -1)
    a.enqueue(1, 10)
    with pytest.raises(TsdfError):
        a.enqueue(1, 10)                     # duplicate id
    with pytest.raises(TsdfError):
        a.release(1)                         # not admitted yet
    a.cancel(1)
    with pytest.raises(TsdfError):
        a.cancel(1)
    assert a.admit() == []
    with pytest.raises(TsdfError):
        Admission(budget_bytes=0, max_active=1)
    with pytest.raises(TsdfError):
        Admission(budget_bytes=10, max_active=0)


class _Model:
    """The admission policy stated plainly: a list in arrival order; admit
    from its front while the front fits the remaining budget and a slot is
    free."""

    def __init__(self, budget, slots):
        self.budget, self.slots = budget, slots
        self.queue, self.active = [], {}

    def admit(self):
        out = []
        while self.queue and len(self.active) < self.slots:
            sid, b = self.queue[0]
            if sum(self.active.values()) + b > self.budget:
                break
            self.queue.pop(0)
            self.active[sid] = b
            out.append(sid)
        return out


def test_matches_policy_model_on_random_traffic():
    rng = np.random.default_rng(3)
    budget, slots = 1000, 7
    a, m = Admission(budget, slots), _Model(budget, slots)
    next_id = 1
    for _ in range(3000):
        op = rng.integers(0, 4)
        if op == 0:
            b = int(rng.integers(1, budget + 1) if rng.uniform() < 0.1 else rng.integers(1, 300))
            a.enqueue(next_id, b)
            m.queue.append((next_id, b))
            next_id += 1
        elif op == 1 and m.active:
            sid = int(rng.choice(sorted(m.active)))
            a.release(sid)
            del m.active[sid]
        elif op == 2 and m.queue and rng.uniform() < 0.2:
            sid = m.queue[int(rng.integers(0, len(m.queue)))][0]
            a.cancel(sid)
            m.queue = [q for q in m.queue if q[0] != sid]
        else:
            assert a.admit() == m.admit()
        st = a.stats()
        assert st["active_bytes"] == sum(m.active.values()) <= budget
        assert st["active"] == len(m.active) <= slots
        assert st["queued"] == len(m.queue)


def test_scene_device_bytes():
    base = dict(voxel_size=0.005, mu=0.02, hash_buckets_log2=16, excess_entries=1 << 12,
                pool_blocks=1 << 14)
    b32 = scene_device_bytes(**base, storage=STORAGE_F32)
    b16 = scene_device_bytes(**base, storage=STORAGE_I16)
    assert b16 == scene_device_bytes(**base, storage=STORAGE_F16)
    assert b32 - b16 == (1 << 14) * 512 * 2              # 4- vs 2-byte sdf per voxel
    assert b16 > (1 << 14) * 512 * 3                     # sdf + weight of the pool at least
    # two sanitised depth buffers (the frame sets)
    assert scene_device_bytes(640, 480, **base, storage=STORAGE_I16) - b16 == 2 * 640 * 480 * 4
    bigger = scene_device_bytes(**{**base, "pool_blocks": 1 << 15}, storage=STORAGE_I16)
    assert bigger - b16 > (1 << 14) * 512 * 3
    with pytest.raises(TsdfError):
        scene_device_bytes(**{**base, "pool_blocks": 0})
