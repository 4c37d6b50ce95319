"""The factor kernel's claim protocol cannot deadlock, checked on the host by
a discrete simulation of W warps over a plan's real schedule
(hylu_export_schedule) with the kernel's rules:

- warps come 4 per block; the first 2 of every block take heavy rows first,
  from a level-ordered queue used only when every heavy row gets such a warp
  at once; any warp that finds the main queue drained also takes from it;
- the main queue is the level-ordered list of rows and tail tasks, and skips
  the heavy rows whenever the heavy queue is in use;
- a row waits for every source node to be complete and, inside a supernode,
  for the diagonal-block step of the row before it; a tail task waits for the
  diagonal-block step of its node's last row;
- a standalone row completes its node; a supernode row publishes its
  diagonal-block step, and its node is complete after its last row (no tail
  tasks) or after the node's last tail task.

The GPU always runs hundreds of blocks; the simulation covers one to a few
blocks, where a wrong claim order would leave every warp waiting."""
import numpy as np
import pytest

from paper_2509_07690_gb300 import Solver, capi, synth

FWARPS, HEAVY_WPB = 4, 2


def _plan(A, **opts):
    s = Solver(A.n, A.rowptr, A.col, A.val, **opts)
    info = s.get_info()
    rp, cp, dr, dc, sn = s.export_perm()
    prp, pci = s.export_pattern()
    order, heavy, task_node = capi.hylu_export_schedule(s.h, A.n, info.ntasks, info.nheavy)
    s.close()
    n = A.n
    node_of = np.repeat(np.arange(len(sn) - 1), np.diff(sn))
    first = sn[node_of]
    # source nodes of every row: its L columns (those below its node)
    srcs = []
    for i in range(n):
        cols = pci[prp[i]:prp[i + 1]]
        srcs.append(set(node_of[cols[cols < first[i]]].tolist()))
    return n, sn, node_of, srcs, order, heavy, task_node


def simulate(plan, blocks):
    n, sn, node_of, srcs, order, heavy, task_node = plan
    nnodes = len(sn) - 1
    ntask = np.bincount(task_node, minlength=nnodes) if len(task_node) else np.zeros(nnodes, int)
    node_size = np.diff(sn)
    nheavy = len(heavy)
    hcap = nheavy if nheavy <= HEAVY_WPB * blocks else 0
    heavy_rank = np.full(n, np.iinfo(np.int32).max)
    heavy_rank[heavy] = np.arange(nheavy)
    done_node = np.zeros(nnodes, bool)
    tasks_done = np.zeros(nnodes, int)
    dready = np.zeros(n, bool)
    hptr = [0]
    mptr = [0]
    nw = blocks * FWARPS
    heavy_open = [(w % FWARPS) < HEAVY_WPB and hcap > 0 for w in range(nw)]
    main_open = [True] * nw
    DONE = -1

    def claim(w):
        if heavy_open[w]:
            h = hptr[0]
            hptr[0] += 1
            if h < hcap:
                return int(heavy[h])
            heavy_open[w] = False
        while main_open[w]:
            qi = mptr[0]
            mptr[0] += 1
            if qi >= len(order):
                main_open[w] = False
                break
            c = int(order[qi])
            if c >= n or hcap == 0 or heavy_rank[c] >= hcap:
                return c
        if hcap > 0:
            h = hptr[0]
            hptr[0] += 1
            if h < hcap:
                return int(heavy[h])
        return DONE

    def ready(c):
        if c >= n:
            D = task_node[c - n]
            return dready[sn[D + 1] - 1]
        D = node_of[c]
        if any(not done_node[S] for S in srcs[c]):
            return False
        return c == sn[D] or dready[c - 1]

    def complete(c):
        if c >= n:
            D = task_node[c - n]
            tasks_done[D] += 1
            if tasks_done[D] == ntask[D]:
                done_node[D] = True
            return
        D = node_of[c]
        if node_size[D] == 1:
            done_node[D] = True
            return
        dready[c] = True
        if ntask[D] == 0 and c == sn[D + 1] - 1:
            done_node[D] = True

    held = [claim(w) for w in range(nw)]
    finished = 0
    total = len(order)
    while True:
        progress = False
        for w in range(nw):
            c = held[w]
            if c != DONE and ready(c):
                complete(c)
                finished += 1
                held[w] = claim(w)
                progress = True
        if all(c == DONE for c in held):
            break
        if not progress:
            stuck = [c for c in held if c != DONE]
            raise AssertionError(f"deadlock with {blocks} block(s): {len(stuck)} warps waiting, "
                                 f"{finished} of {total} tasks done")
    assert finished == total
    assert done_node.all()
    return hcap


CASES = [
    ("grid5_16", lambda: synth.grid5(16), {}),
    ("convdiff_10_nd", lambda: synth.convdiff3d(10), {"ordering": 1}),
    ("aniso_24_nd", lambda: synth.aniso9(24), {"ordering": 1}),
    ("circuit_2500", lambda: synth.circuit(2500, seed=31), {}),
    ("circuit_4000", lambda: synth.circuit(4000, seed=77), {}),
    ("circuit_4000_nd", lambda: synth.circuit(4000, seed=77), {"ordering": 1}),
]


@pytest.mark.parametrize("name,make,opts", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("blocks", [1, 2, 3, 16])
def test_claim_protocol_completes(name, make, opts, blocks):
    plan = _plan(make(), **opts)
    simulate(plan, blocks)


@pytest.mark.parametrize("ratio,blocks", [(90.0, 8), (90.0, 9), (90.0, 3), (32.0, 100)])
def test_heavy_queue_exercised(ratio, blocks):
    """The heavy-row queue in use (every heavy row fits the heavy warps) or
    switched off (too few blocks): the simulation completes either way."""
    plan = _plan(synth.circuit(20000, seed=77), heavy_ratio=ratio)
    nheavy = len(plan[5])
    assert nheavy > 0
    hcap = simulate(plan, blocks)
    assert hcap == (nheavy if nheavy <= HEAVY_WPB * blocks else 0)


def test_simulation_detects_a_wrong_order():
    """The simulation is not vacuous: the same plan claimed in reverse level
    order leaves every warp of one block waiting on unclaimed rows."""
    n, sn, node_of, srcs, order, heavy, task_node = _plan(synth.grid5(16))
    bad = (n, sn, node_of, srcs, order[::-1].copy(), heavy, task_node)
    with pytest.raises(AssertionError, match="deadlock"):
        simulate(bad, 1)
