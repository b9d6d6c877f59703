"""Specimen sharding across ranks (host logic of the multi-GPU batch path),
checked on CPU: a brute-force optimum on small cases, the 4/3 bound on the
96-specimen batch, and two gloo ranks that compute their shards independently
and find them disjoint and complete."""
import itertools
import os
import tempfile

import numpy as np
import pytest

from paper_2604_03411_gb300 import inputs as I
from paper_2604_03411_gb300 import shard as S


def loads(parts, costs):
    return [sum(costs[i] for i in p) for p in parts]


def test_partition_covers_and_is_deterministic():
    rng = np.random.default_rng(0)
    costs = list(rng.integers(1, 100, size=37).astype(float))
    for w in (1, 2, 3, 8, 40):
        parts = S.partition(costs, w)
        assert len(parts) == w
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        assert parts == S.partition(costs, w)


def test_partition_within_four_thirds_of_brute_force():
    rng = np.random.default_rng(1)
    for trial in range(20):
        n = int(rng.integers(2, 9))
        w = int(rng.integers(2, 4))
        costs = list(rng.integers(1, 50, size=n).astype(float))
        best = min(max(sum(c for c, r in zip(costs, asg) if r == k) for k in range(w))
                   for asg in itertools.product(range(w), repeat=n))
        got = max(loads(S.partition(costs, w), costs))
        assert got <= (4.0 / 3.0 - 1.0 / (3 * w)) * best + 1e-9, (costs, w, got, best)


def test_partition_of_the_96_specimen_batch():
    probs = I.config5()
    costs = [S.specimen_cost(p) for p in probs]
    total = sum(costs)
    for w in (2, 4, 8):
        ld = loads(S.partition(costs, w), costs)
        lower = max(total / w, max(costs))
        assert max(ld) <= (4.0 / 3.0) * lower
        assert max(ld) <= 1.05 * total / w            # many small items: close to perfect


def _rank(rank, world, path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"file://{path}.init")
    costs = [float(c) for c in np.random.default_rng(7).integers(10, 500, size=96)]
    mine = S.partition(costs, world)[rank]
    got = [None] * world
    dist.all_gather_object(got, mine)
    flat = sorted(i for p in got for i in p)
    ok = flat == list(range(96)) and all(set(a).isdisjoint(b) for a, b in itertools.combinations(got, 2))
    with open(f"{path}.{rank}", "w") as f:
        f.write("ok" if ok else f"bad {got}")
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_split():
    mp = pytest.importorskip("torch.multiprocessing")
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "shard")
        mp.spawn(_rank, args=(2, path), nprocs=2, join=True)
        for r in range(2):
            assert open(f"{path}.{r}").read() == "ok"
