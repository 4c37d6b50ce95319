"""Random plans through every host check at once: random sparse matrices of
four kinds (scattered, banded, with dense hub rows and columns, dense
diagonal blocks), each under a random ordering (AMD, nested dissection,
natural, AUTO) and supernode cap.  Per plan: pattern, partition and flop
count equal the oracle's; the checkpoint image re-saves to the same bytes;
the value-scatter map and tail tasks are consistent; the substitution
schedules pass their dependency, count and replay checks; and the factor
kernel's claim protocol completes with one and three blocks."""
import numpy as np
import pytest

import oracle
from paper_2509_07690_gb300 import Solver, synth
from plan_image import PlanImage
import test_plan_tables as tables
import test_schedule as claims
import test_substitution_schedule as subst


def _matrix(rng, kind):
    n = int(rng.integers(2, 260))
    a = np.where(rng.random((n, n)) < rng.uniform(0.5, 6.0) / n, rng.uniform(-1, 1, (n, n)), 0.0)
    if kind == "banded":
        bw = int(rng.integers(1, 8))
        extra = np.where(rng.random((n, n)) < 0.5, rng.uniform(-1, 1, (n, n)), 0.0)
        a = np.triu(np.tril(a + extra, bw), -bw)
    elif kind == "hubs":
        for h in rng.choice(n, int(rng.integers(1, min(4, n) + 1)), replace=False):
            a[h, :] = np.where(rng.random(n) < 0.5, rng.uniform(-1, 1, n), a[h, :])
            a[:, h] = np.where(rng.random(n) < 0.5, rng.uniform(-1, 1, n), a[:, h])
    elif kind == "blocks":
        off = 0
        while off < n:
            b = min(int(rng.integers(1, 20)), n - off)
            a[off:off + b, off:off + b] = rng.uniform(-1, 1, (b, b))
            off += b
    a[np.arange(n), np.arange(n)] = np.abs(a).sum(axis=1) + rng.uniform(0.5, 1.5, n)
    r, c = np.nonzero(a)
    return synth.from_coo(n, r, c, a[r, c])


@pytest.mark.parametrize("seed", range(120))
def test_random_plan_passes_every_host_check(seed):
    rng = np.random.default_rng(31000 + seed)
    kind = ("scattered", "banded", "hubs", "blocks")[seed % 4]
    A = _matrix(rng, kind)
    opts = {"ordering": int(rng.choice([0, 1, 2, 4])), "sn_max": int(rng.choice([1, 3, 8, 64, 256])),
            "heavy_ratio": float(rng.choice([0.0, 1.0, 32.0]))}
    s = Solver(A.n, A.rowptr, A.col, A.val, **opts)
    rp, cp, dr, dc, sn = s.export_perm()
    o = oracle.Oracle(A.n, A.rowptr, A.col, A.val, rp, cp, dr, dc, sn_max=opts["sn_max"], numeric=False)
    prp, pci = s.export_pattern()
    assert np.array_equal(o.sn_start, sn)
    assert np.array_equal(o.padded.rowptr, prp) and np.array_equal(o.padded.col, pci)
    assert s.info.flops == o.flops[0]
    image = s.save()
    s.close()
    t = Solver.load(image)
    assert t.save() == image
    t.close()
    img = PlanImage(image)
    tables.check_scatter(img)
    tables.check_tasks(img)
    subst.check_dependencies(img)
    for k in subst.KINDS:
        subst.check_counts(img, k)
        subst.simulate(img, k)
    plan = claims._plan(A, **opts)
    for blocks in (1, 3):
        claims.simulate(plan, blocks)
