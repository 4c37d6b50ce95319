"""Host tables of the precision form's tensor-core sup-sup update (HYLU
Sec. 2.2, Fig. 1c), rebuilt here by brute force from the exported padded
pattern and compared entry by entry: the destination set (large supernodes
and everything downstream of one), each destination's union of L columns,
the union position of every L slot, the (N tile, source segment, tail
range) triples that say which source tail entries land in which tile, the K
chunks of every tile, the GEMM task list, and the claim order (every task
after everything it waits on)."""
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
    is_gd = np.zeros(nn, bool)
    for D in range(nn):
        is_gd[D] = (sn[D + 1] - sn[D]) >= min_rows or any(is_gd[S] for S in src[D])
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
    assert np.array_equal(G["gd_node"], gd)
    lslot0 = np.concatenate([[0], np.cumsum([len(x) for x in B["lcols"]])])
    a_off = 0
    for g, D in enumerate(gd):
        r, e = sn[D], sn[D + 1] - 1
        sD = e - r + 1
        lc = np.unique(np.concatenate([B["lcols"][i] for i in range(r, e + 1)] + [np.zeros(0, np.int64)]))
        got_lc = G["lc_cols"][G["gd_lc_off"][g]:G["gd_lc_off"][g + 1]]
        assert np.array_equal(got_lc, lc)
        K = len(lc)
        assert G["gd_K"][g] == K and G["gd_Kp"][g] == -(-K // TK) * TK
        assert G["gd_Mp"][g] == -(-sD // TM) * TM
        assert G["gd_a_off"][g] == a_off
        a_off += G["gd_Mp"][g] * G["gd_Kp"][g]
        for i in range(r, e + 1):
            pos = G["lu_pos"][lslot0[i]:lslot0[i + 1]]
            assert np.array_equal(lc[pos], B["lcols"][i])
        ucols = np.concatenate([np.arange(r, e + 1), B["tail"][D]])
        ntiles = -(-len(ucols) // TN)
        assert G["gd_ntiles"][g] == ntiles
        uidx = {int(c): x for x, c in enumerate(ucols)}
        # every (tile, union column, tail entry) the product needs, by brute force
        want = set()
        for k in lc:
            S = int(node_of[k])
            for j, c in enumerate(B["tail"][S]):
                if c >= r:
                    want.add((uidx[int(c)] // TN, int(k), j))
        got = set()
        for nt in range(ntiles):
            pair = G["gd_tile_base"][g] + nt
            t0, t1 = G["pr_tri_off"][pair], G["pr_tri_off"][pair + 1]
            for t in range(t0, t1):
                u0, ln, S = G["tri_u0"][t], G["tri_len"][t], G["tri_node"][t]
                assert lc[u0] == sn[S] and ln == sn[S + 1] - sn[S]
                for j in range(G["tri_jlo"][t], G["tri_jhi"][t]):
                    assert uidx[int(B["tail"][S][j])] // TN == nt
                    for k in range(sn[S], sn[S + 1]):
                        got.add((nt, int(k), j))
            # chunks: exactly those overlapping a triple, each with its triples
            c0, c1 = G["pr_ck_off"][pair], G["pr_ck_off"][pair + 1]
            want_ck = sorted({kc for t in range(t0, t1)
                              for kc in range(G["tri_u0"][t] // TK, (G["tri_u0"][t] + G["tri_len"][t] - 1) // TK + 1)})
            assert list(G["ck_kc"][c0:c1]) == want_ck
            for q in range(c0, c1):
                kc = G["ck_kc"][q]
                over = [t for t in range(t0, t1)
                        if G["tri_u0"][t] < (kc + 1) * TK and G["tri_u0"][t] + G["tri_len"][t] > kc * TK]
                assert list(range(G["ck_t0"][q], G["ck_t1"][q])) == over
        assert got == want, (name, D)
    # GEMM tasks: every (destination, M tile, N tile) once, levels ascending
    tasks = sorted(zip(G["task_gd"], G["task_mt"], G["task_nt"]))
    want_tasks = sorted((g, mt, nt) for g in range(len(gd)) for mt in range(G["gd_Mp"][g] // TM)
                        for nt in range(G["gd_ntiles"][g]))
    assert tasks == want_tasks
    assert np.all(np.diff(G["task_level"]) >= 0)
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
    gemm_level = {int(g): int(l) for g, l in zip(G["task_gd"], G["task_level"])}

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
    for D, g in gd_of.items():
        r, e = sn[D], sn[D + 1] - 1
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
