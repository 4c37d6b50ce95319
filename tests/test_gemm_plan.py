"""Host tables of the precision form's tensor-core sup-sup update (HYLU
Sec. 2.2, Fig. 1c), rebuilt here by brute force from the exported padded
pattern and compared entry by entry: the destination set (the supernodes of
at least gemm_min_rows rows),
the (destination, large source) pairs with their A columns, tail ranges and
U-column maps, the pair named at each L slot, the GEMM task list, and the
claim order (every task after everything it waits on)."""
import numpy as np
import pytest

from paper_2509_07690_gb300 import Solver, capi, synth

TN, TK, TM = 64, 32, 128


def _cases():
    rng = np.random.default_rng(3)
    a = rng.standard_normal((90, 90)) * (rng.random((90, 90)) < 0.08) + 8 * np.eye(90)
    r, c = np.nonzero(a)
    yield "random_90", synth.from_coo(90, r, c, a[r, c]), {}
    yield "convdiff_8_nd", synth.convdiff3d(8), {"ordering": 1}
    yield "grid5_20_amd", synth.grid5(20), {}
    yield "circuit_1500", synth.circuit(1500, seed=4), {}
    yield "aniso_24_nd", synth.aniso9(24), {"ordering": 1}


CASES = list(_cases())


def _brute(s, min_rows):
    n = s.n
    rp, ci = s.export_pattern()
    _, _, _, _, sn = s.export_perm()
    nn = len(sn) - 1
    node_of = np.repeat(np.arange(nn), np.diff(sn))
    rows = [ci[rp[i]:rp[i + 1]] for i in range(n)]
    lcols = [rows[i][rows[i] < sn[node_of[i]]] for i in range(n)]
    tail = [rows[sn[S]][rows[sn[S]] >= sn[S + 1]] for S in range(nn)]
    src = [sorted({int(node_of[k]) for i in range(sn[D], sn[D + 1]) for k in lcols[i]}) for D in range(nn)]
    is_gd = np.diff(sn) >= min_rows
    return dict(n=n, sn=sn, node_of=node_of, lcols=lcols, tail=tail, src=src, is_gd=is_gd)


@pytest.mark.parametrize("min_rows", [4, 16])
@pytest.mark.parametrize("name,A,opts", CASES, ids=[c[0] for c in CASES])
def test_gemm_plan_matches_brute_force(name, A, opts, min_rows):
    s = Solver(A.n, A.rowptr, A.col, A.val, **opts)
    G = capi.hylu_export_gemm_plan(s.h, min_rows, A.n)
    B = _brute(s, min_rows)
    sn, node_of = B["sn"], B["node_of"]
    gd = np.nonzero(B["is_gd"])[0]
    assert G["ngd"] == len(gd)
    if len(gd) == 0:
        s.close()
        return
    min_src = min(16, max(2, min_rows))
    assert G["min_src"] == min_src
    assert np.array_equal(G["gd_node"], gd)
    lslot0 = np.concatenate([[0], np.cumsum([len(x) for x in B["lcols"]])])
    want_pairs = []
    a_off = 0
    for g, D in enumerate(gd):
        r, e = sn[D], sn[D + 1] - 1
        sD = e - r + 1
        ucols = np.concatenate([np.arange(r, e + 1), B["tail"][D]])
        uidx = {int(c): x for x, c in enumerate(ucols)}
        kp = 0
        for S in B["src"][D]:
            ln = sn[S + 1] - sn[S]
            T = B["tail"][S]
            jr = int(np.searchsorted(T, r))
            if ln < min_src or jr == len(T):
                continue
            need = sum(1 for i in range(r, e + 1) if sn[S] in set(B["lcols"][i].tolist()))
            want_pairs.append((g, S, kp, ln, jr, len(T) - jr, need, [uidx[int(c)] for c in T[jr:]]))
            kp += -(-ln // TK) * TK
        assert G["gd_Kp"][g] == kp and G["gd_Mp"][g] == -(-sD // TM) * TM
        assert G["gd_a_off"][g] == a_off
        a_off += G["gd_Mp"][g] * kp
    assert G["a_elems"] == a_off
    assert G["npair"] == len(want_pairs)
    for p, (g, S, u0, ln, jr, nj, need, xm) in enumerate(want_pairs):
        got = (G["pair_gd"][p], G["pair_src"][p], G["pair_u0"][p], G["pair_len"][p], G["pair_jr"][p],
               G["pair_nj"][p], G["pair_need"][p])
        assert got == (g, S, u0, ln, jr, nj, need), p
        x0 = G["pair_x_off"][p]
        assert list(G["xmap"][x0:x0 + nj]) == xm
    # the first L slot of every large source segment in a destination row
    # names its pair; no other slot does
    pair_of = {(int(G["pair_gd"][p]), int(G["pair_src"][p])): p for p in range(G["npair"])}
    gd_of = {int(D): g for g, D in enumerate(gd)}
    want_slot = np.full(G["nl"], -1)
    for i in range(A.n):
        D = int(node_of[i])
        if D not in gd_of:
            continue
        for t, k in enumerate(B["lcols"][i]):
            S = int(node_of[k])
            if k == sn[S] and (gd_of[D], S) in pair_of:
                want_slot[lslot0[i] + t] = pair_of[(gd_of[D], S)]
    assert np.array_equal(G["gd_slot"], want_slot)
    # GEMM tasks: every (pair, M tile, tail tile) once, levels ascending, and
    # the per-destination counts
    tasks = sorted(zip(G["task_pair"], G["task_mt"], G["task_jt"]))
    want_tasks = sorted((p, mt, jt) for p, w in enumerate(want_pairs)
                        for mt in range(G["gd_Mp"][w[0]] // TM) for jt in range(-(-w[5] // TN)))
    assert tasks == want_tasks
    assert np.all(np.diff(G["task_level"]) >= 0)
    cnt = np.bincount(G["pair_gd"][G["task_pair"]], minlength=len(gd))
    assert np.array_equal(G["gd_ntask"], cnt)
    s.close()


@pytest.mark.parametrize("name,A,opts", CASES, ids=[c[0] for c in CASES])
def test_gemm_claim_order_respects_dependencies(name, A, opts):
    """Every queued task comes after everything it waits on: a row's walk
    after its sources complete, a GEMM tile (its own queue, by level) after
    every walk of its destination, a diag step after the destination's tiles
    and the previous row's step, a tail task after the node's last step."""
    s = Solver(A.n, A.rowptr, A.col, A.val, **opts)
    G = capi.hylu_export_gemm_plan(s.h, 8, A.n)
    B = _brute(s, 8)
    if G["ngd"] == 0:
        s.close()
        pytest.skip("no destination")
    n = A.n
    info = s.get_info()
    _, _, task_node = capi.hylu_export_schedule(s.h, n, info.ntasks, info.nheavy)
    ntask = info.ntasks - n
    nd = G["ndiag"]
    order = G["row_order"]
    assert sorted(order) == list(range(n + ntask + nd))
    where = np.empty(len(order), np.int64)
    where[order] = np.arange(len(order))
    sn, node_of = B["sn"], B["node_of"]
    gd_of = {int(D): g for g, D in enumerate(G["gd_node"])}
    diag_of = {int(i): d for d, i in enumerate(G["diag_row"])}
    tasks_of = {}
    for t, D in enumerate(task_node):
        tasks_of.setdefault(int(D), []).append(n + t)
    gemm_level = {int(G["pair_gd"][p]): int(l) for p, l in zip(G["task_pair"], G["task_level"])}

    def complete(S):
        """Queue positions whose end completes node S."""
        if S in tasks_of:
            return [where[x] for x in tasks_of[S]]
        e = sn[S + 1] - 1
        return [where[n + ntask + diag_of[e]]] if S in gd_of else [where[e]]

    for i in range(n):
        D = int(node_of[i])
        for S in {int(node_of[k]) for k in B["lcols"][i]}:
            assert where[i] > max(complete(S)), (i, S)
        if D not in gd_of and i > sn[D]:
            assert where[i] > where[i - 1]
        assert G["walk_level"][i] >= 0
    for D, g in gd_of.items():
        r, e = sn[D], sn[D + 1] - 1
        if g not in gemm_level:
            continue
        lg = gemm_level[g]
        assert all(G["walk_level"][i] < lg for i in range(r, e + 1))
        for i in range(r, e + 1):
            assert G["diag_level"][i] > lg
            if i > r:
                assert where[n + ntask + diag_of[i]] > where[n + ntask + diag_of[i - 1]]
        for x in tasks_of.get(D, []):
            assert where[x] > where[n + ntask + diag_of[e]]
    s.close()


def test_no_destination_below_threshold_or_when_disabled():
    A = synth.grid5(6)
    s = Solver(A.n, A.rowptr, A.col, A.val)
    assert capi.hylu_export_gemm_plan(s.h, 0, A.n)["ngd"] == 0
    assert capi.hylu_export_gemm_plan(s.h, 10_000, A.n)["ngd"] == 0
    s.close()
