"""Learned prescreen and incremental local search on the GPU: the kept moves
are the lowest predicted deltas (checked against the oracle's features and
MLP), the incremental cost update equals a full re-evaluation, and a
screened search improves plans exactly (costs re-checked by the oracle)."""
import numpy as np
import pytest

import oracle
import wh_gen
from paper_2110_13693_gb300 import search

pytestmark = pytest.mark.gpu


def setup(wh, inst, per_plan=True):
    n = inst.n_plans
    smap = np.tile(inst.slot_map, (n, 1)).ravel().astype(np.int32) if per_plan else inst.slot_map
    lay = wh.Layout.of(inst.layout)
    prob = wh.to_device(inst, slot_map=smap, slot_map_stride=inst.n_sku if per_plan else 0)
    costs = wh.evaluate(lay, prob)
    return lay, prob, costs


def moves_for(inst, seed, step, M):
    import torch
    mv = wh_gen.gen_moves(seed, step, inst, M)
    mv[..., 3] = np.arange(inst.n_plans)[:, None]
    return torch.as_tensor(mv.reshape(-1, 4)).cuda()


def test_incremental_costs_equal_full_refresh(gpu_lib):
    import torch
    wh = gpu_lib
    inst = wh_gen.paperscale(seed=21, n_plans=24)
    a = setup(wh, inst)
    b = setup(wh, inst)
    for step in range(4):
        mv = moves_for(inst, 3, step, 32)
        ra = a[0].ls_step(a[1], a[2], mv, 32, 24)
        rb = b[0].ls_step(b[1], b[2], mv, 32, 24, refresh=True)
        torch.cuda.synchronize()
        assert torch.equal(ra, rb)
        for x, y in ((a[2].tour_rr, b[2].tour_rr), (a[2].tour_s, b[2].tour_s)):
            assert torch.equal(x[:a[1].n_tours], y[:b[1].n_tours])
        assert torch.equal(a[2].plan_rr[:24], b[2].plan_rr[:24]) and torch.equal(a[2].plan_s[:24], b[2].plan_s[:24])
    assert a[0].status() == 0


def moved_tours(inst, smap, mv):
    """Changed tours of a move as (new pick list, old tour index) pairs (Python, from the definition)."""
    typ, x, y, p = (int(v) for v in mv)
    t0, t1 = inst.plan_tour_off[p], inst.plan_tour_off[p + 1]
    tours = {t: inst.order_seq[inst.tour_off[t]:inst.tour_off[t + 1]].tolist() for t in range(t0, t1)}
    where = {o: t for t, os in tours.items() for o in os}
    lines = lambda os, m: [m[s] for o in os for s in inst.line_sku[inst.order_off[o]:inst.order_off[o + 1]]]
    if typ == 0:
        ta, tb = where[x], where[y]
        return [(lines([y if o == x else o for o in tours[ta]], smap), ta),
                (lines([x if o == y else o for o in tours[tb]], smap), tb)]
    if typ == 1:
        ta, tb = where[x], t0 + y
        return [(lines([o for o in tours[ta] if o != x], smap), ta), (lines(tours[tb] + [x], smap), tb)]
    m2 = smap.copy()
    if typ == 2:
        m2[x], m2[y] = m2[y], m2[x]
        skus = {x, y}
    else:                                   # relocation of SKU x to the empty location y
        m2[x] = y
        skus = {x}
    hit = {where[o] for o in range(inst.n_orders) if o in where and
           (set(inst.line_sku[inst.order_off[o]:inst.order_off[o + 1]].tolist()) & skus)}
    return [(lines(tours[t], m2), t) for t in sorted(hit)]


@pytest.mark.parametrize("which", ["tiny", "paperscale"])
def test_screen_task_features_bit_exact(gpu_lib, which):
    """Every counted task's feature row (its changed tour under the move,
    rebuilt here from the move's definition) equals the oracle's features bit
    for bit: a tiny layout (16-bit keys, one task per thread) and paper scale
    (32-bit keys; tasks over 64 lines go to the warp-per-task kernel)."""
    import torch
    wh = gpu_lib
    tiny = which == "tiny"
    inst = wh_gen.tiny(seed=22, n_plans=5) if tiny else wh_gen.paperscale(seed=21, n_plans=3)
    lay, prob, costs = setup(wh, inst)
    sg = wh.Surrogate(3)
    M = 32 if tiny else 24
    mv = moves_for(inst, 5, 0, M)
    lay.screen(sg, prob, mv, M, 4, 8 if tiny else 0)
    torch.cuda.synchronize()
    assert lay.status() == 0
    tasks, counted, rows = lay.screen_trace()
    tasks, counted = tasks.cpu().numpy(), counted.cpu().numpy()
    bits = rows.view(torch.int16).cpu().numpy()
    mvn = mv.cpu().numpy()
    changed, n_checked, n_long = {}, 0, 0
    for i in range(tasks.shape[0]):
        if counted[i, 0] != 0:
            continue
        m, t = int(tasks[i, 0]), int(tasks[i, 1])
        if m not in changed:
            changed[m] = {t_old: locs for locs, t_old in moved_tours(inst, inst.slot_map, mvn[m])}
        locs = changed[m][t]
        want = torch.from_numpy(oracle.bf16(oracle.features(inst.layout, locs))).to(torch.bfloat16)
        assert np.array_equal(bits[i], want.view(torch.int16).numpy()), (which, i, m, t)
        n_checked += 1
        n_long += len(locs) > 64
    assert n_checked >= 40
    if not tiny:
        assert n_long >= 5
    # any other call on the layout leaves no trace
    lay.eval_moves(prob, costs, mv)
    torch.cuda.synchronize()
    assert lay.screen_trace() is None
    sg.close()
    lay.close()


@pytest.mark.parametrize("which", ["paperscale", "relocations"])
def test_screen_eval_equals_screen_then_eval_moves(gpu_lib, which):
    """The one-call prescreen and exact re-score (the exact pass on the
    prescreen's index) gives the kept moves, deltas and statuses that the
    prescreen followed by eval_moves on the kept moves gives, and applying them
    leaves the same plans, costs and changed-tour flags, step after step: paper
    scale (per-plan slottings, all order and SKU moves, tasks over 64 lines)
    and relocations into empty locations."""
    import torch
    wh = gpu_lib
    if which == "paperscale":
        inst = wh_gen.paperscale(seed=21, n_plans=12)
        M, max_orders = 32, 24
        moves = lambda step: moves_for(inst, 7, step, M)
    else:
        base = wh_gen.tiny(seed=24, n_plans=4)
        lay_d = wh_gen.Layout(20, 30)
        smap = np.random.default_rng(24).permutation(lay_d.n_loc)[:base.n_sku].astype(np.int32)
        inst = wh_gen.Instance(lay_d, base.n_sku, base.order_off, base.line_sku, smap, base.plan_tour_off,
                               base.tour_off, base.order_seq)
        M, max_orders = 32, 8

        def moves(step):
            mv = np.concatenate([wh_gen.gen_moves(6, step, inst, M // 2),
                                 wh_gen.gen_relocations(7, step, inst, M // 2)], axis=1)
            mv[..., 3] = np.arange(inst.n_plans)[:, None]
            return torch.as_tensor(mv.reshape(-1, 4)).cuda()
    a, b = setup(wh, inst), setup(wh, inst)
    if which != "paperscale":
        a[0].occupancy(a[1])
        b[0].occupancy(b[1])
    sg = wh.Surrogate(3)
    keep = 4
    ca, cb = search.new_cache(a[1]), search.new_cache(b[1])
    for step in range(3):
        mv = moves(step)
        kept_a, d_a, s_a = a[0].screen_eval(sg, a[1], a[2], mv, M, keep, max_orders, y_tour=ca[0], changed=ca[1])
        kept_b = b[0].screen(sg, b[1], mv, M, keep, max_orders, y_tour=cb[0], changed=cb[1])
        d_b, s_b = b[0].eval_moves(b[1], b[2], kept_b, max_orders)
        torch.cuda.synchronize()
        assert torch.equal(kept_a, kept_b) and torch.equal(d_a, d_b) and torch.equal(s_a, s_b), step
        assert (s_a == 0).sum() > 0
        ra = a[0].apply_scored(a[1], a[2], kept_a, keep, d_a, s_a, changed=ca[1])
        rb = b[0].ls_step(b[1], b[2], kept_b, keep, max_orders, changed=cb[1])
        torch.cuda.synchronize()
        assert torch.equal(ra, rb) and (ra >= 0).sum() > 0
        for x, y in ((a[1].order_seq, b[1].order_seq), (a[1].tour_off, b[1].tour_off),
                     (a[1].slot_map, b[1].slot_map), (ca[1], cb[1])):
            assert torch.equal(x, y)
        n_t, n_p = a[1].n_tours, a[1].n_plans
        for x, y in ((a[2].tour_s[:n_t], b[2].tour_s[:n_t]), (a[2].tour_rr[:n_t], b[2].tour_rr[:n_t]),
                     (a[2].plan_s[:n_p], b[2].plan_s[:n_p]), (a[2].plan_rr[:n_p], b[2].plan_rr[:n_p])):
            assert torch.equal(x, y)
    # the incrementally updated costs are the exact costs of the edited plans
    fresh = wh.evaluate(a[0], a[1])
    torch.cuda.synchronize()
    assert torch.equal(fresh.plan_rr[:a[1].n_plans], a[2].plan_rr[:a[1].n_plans])
    assert torch.equal(fresh.plan_s[:a[1].n_plans], a[2].plan_s[:a[1].n_plans])
    assert a[0].status() == 0 and b[0].status() == 0
    sg.close()


def test_screen_keeps_lowest_predicted_deltas(gpu_lib):
    import torch
    wh = gpu_lib
    inst = wh_gen.tiny(seed=22, n_plans=5)
    lay, prob, costs = setup(wh, inst)
    sg = wh.Surrogate(3)
    X, t = search.training_set(wh, lay, prob, costs, inst.layout)
    search.train(sg, X, t, 60, 256, 3e-3)
    M, keep = 32, 4
    mv = moves_for(inst, 5, 0, M)
    kept = lay.screen(sg, prob, mv, M, keep, 8).cpu().numpy().reshape(inst.n_plans, keep, 4)
    params = wh.unpack_params(sg.params()[0])
    w = {k: (oracle.bf16(v) if k in ("w1", "w2") else v) for k, v in params.items()}
    pred = lambda locs: oracle.mlp_forward(w, oracle.bf16(oracle.features(inst.layout, locs))[None])[0]
    d, st = oracle.eval_moves(inst, mv.cpu().numpy(), 8, 0, slot_map=np.tile(inst.slot_map, (5, 1)).ravel(),
                              slot_map_stride=inst.n_sku)
    smap = inst.slot_map
    old = {}
    for p in range(inst.n_plans):
        scores = {}
        for k in range(M):
            m = p * M + k
            if st[m] != 0:
                continue
            sc = 0.0
            for locs, t_old in moved_tours(inst, smap, mv[m].cpu().numpy()):
                if t_old not in old:
                    orig = [smap[s] for o in inst.order_seq[inst.tour_off[t_old]:inst.tour_off[t_old + 1]]
                            for s in inst.line_sku[inst.order_off[o]:inst.order_off[o + 1]]]
                    old[t_old] = pred(orig)
                sc += pred(locs) - old[t_old]
            scores[k] = sc
        order = sorted(scores.values())
        kth = order[min(keep, len(order)) - 1] if order else None
        moves_p = mv[p * M:(p + 1) * M].cpu().numpy().tolist()
        for j in range(keep):
            if j >= len(scores):
                assert kept[p, j, 0] == 9
                continue
            k = moves_p.index(kept[p, j].tolist())
            assert scores[k] <= kth + 1e-3 * max(1.0, abs(kth)), (p, j, scores[k], kth)
    sg.close()
    lay.close()


def test_screened_search_improves_exactly(gpu_lib):
    import torch
    wh = gpu_lib
    inst = wh_gen.paperscale(seed=23, n_plans=16)
    lay, prob, costs = setup(wh, inst)
    sg = wh.Surrogate(4)
    X, t = search.training_set(wh, lay, prob, costs, inst.layout)
    search.train(sg, X, t, 150, 1024, 2e-3)
    start = costs.plan_rr[:16].clone()
    trace = search.run_search(wh, lay, prob, costs, lambda s: moves_for(inst, 8, s, 64), 4, 64, 24, 0,
                              sg=sg, keep=search.keep_count(64))
    assert (costs.plan_rr[:16] <= start).all() and trace[-1][1] <= int(start.min().item())
    # the incrementally kept costs are the exact costs of the edited plans
    cur = wh_gen.Instance(inst.layout, inst.n_sku, inst.order_off, inst.line_sku, prob.slot_map.cpu().numpy(),
                          inst.plan_tour_off, prob.tour_off.cpu().numpy(), prob.order_seq.cpu().numpy())
    want = oracle.eval_plans(cur, slot_map=cur.slot_map, slot_map_stride=inst.n_sku)
    assert np.array_equal(costs.plan_rr[:16].cpu().numpy(), want[3])
    assert np.array_equal(costs.tour_rr[:prob.n_tours].cpu().numpy(), want[1])
    assert lay.status() == 0
    sg.close()
    lay.close()


def test_prediction_cache_matches_full_recompute(gpu_lib):
    """Screening with the tour-prediction cache (only the tours the previous
    step rewrote are re-predicted) keeps exactly the moves that screening
    with every tour re-predicted keeps, step after step."""
    import torch
    wh = gpu_lib
    inst = wh_gen.paperscale(seed=24, n_plans=12)
    lay, prob, costs = setup(wh, inst)
    lay2, prob2, costs2 = setup(wh, inst)
    sg = wh.Surrogate(5)
    X, t = search.training_set(wh, lay, prob, costs, inst.layout)
    search.train(sg, X, t, 60, 1024, 2e-3)
    y_tour, changed = search.new_cache(prob)
    for step in range(4):
        mv = moves_for(inst, 9, step, 32)
        ka = lay.screen(sg, prob, mv, 32, 4, 24, y_tour=y_tour, changed=changed)
        kb = lay2.screen(sg, prob2, mv, 32, 4, 24)
        assert torch.equal(ka, kb), step
        assert int(changed.sum().item()) == 0
        lay.ls_step(prob, costs, ka, 4, 24, changed=changed)
        lay2.ls_step(prob2, costs2, kb, 4, 24)
        assert torch.equal(costs.plan_rr[:12], costs2.plan_rr[:12])
        # unflagged entries hold the current tours' predictions
        fresh = sg.predict(wh.features(lay2, prob2))
        keep = changed[:prob.n_tours] == 0
        assert torch.equal(y_tour[:prob.n_tours][keep], fresh[keep])
        assert int(changed.sum().item()) > 0
    assert lay.status() == 0 and lay2.status() == 0 and sg.status() == 0
    sg.close()
    lay.close()
    lay2.close()


def test_screen_and_search_with_relocations(gpu_lib):
    """Relocations into empty locations mixed into the screened moves (tiny's
    orders on a half-empty 20 x 30 layout): the kept moves are the lowest
    predicted deltas, and screened steps keep exact costs and occupancy bits."""
    import torch
    wh = gpu_lib
    base = wh_gen.tiny(seed=24, n_plans=4)
    lay_d = wh_gen.Layout(20, 30)
    rng = np.random.default_rng(24)
    smap = rng.permutation(lay_d.n_loc)[:base.n_sku].astype(np.int32)
    inst = wh_gen.Instance(lay_d, base.n_sku, base.order_off, base.line_sku, smap, base.plan_tour_off,
                           base.tour_off, base.order_seq)
    lay, prob, costs = setup(wh, inst)
    lay.occupancy(prob)
    sg = wh.Surrogate(5)
    X, t = search.training_set(wh, lay, prob, costs, inst.layout)
    search.train(sg, X, t, 60, 256, 3e-3)
    M, keep = 32, 4

    def mixed(step):
        mv = np.concatenate([wh_gen.gen_moves(6, step, inst, M // 2), wh_gen.gen_relocations(7, step, inst, M // 2)],
                            axis=1)
        mv[..., 3] = np.arange(inst.n_plans)[:, None]
        return torch.as_tensor(mv.reshape(-1, 4)).cuda()

    mv = mixed(0)
    kept = lay.screen(sg, prob, mv, M, keep, 8).cpu().numpy().reshape(inst.n_plans, keep, 4)
    params = wh.unpack_params(sg.params()[0])
    w = {k: (oracle.bf16(v) if k in ("w1", "w2") else v) for k, v in params.items()}
    pred = lambda locs: oracle.mlp_forward(w, oracle.bf16(oracle.features(inst.layout, locs))[None])[0]
    maps = np.tile(smap, (inst.n_plans, 1))
    d, st = oracle.eval_moves(inst, mv.cpu().numpy(), 8, 0, slot_map=maps.ravel(), slot_map_stride=inst.n_sku)
    assert ((mv[:, 0].cpu().numpy() == 3) & (st == 0)).sum() > 10
    old = {}
    for p in range(inst.n_plans):
        scores = {}
        for k in range(M):
            m = p * M + k
            if st[m] != 0:
                continue
            sc = 0.0
            for locs, t_old in moved_tours(inst, smap, mv[m].cpu().numpy()):
                if t_old not in old:
                    orig = [smap[s] for o in inst.order_seq[inst.tour_off[t_old]:inst.tour_off[t_old + 1]]
                            for s in inst.line_sku[inst.order_off[o]:inst.order_off[o + 1]]]
                    old[t_old] = pred(orig)
                sc += pred(locs) - old[t_old]
            scores[k] = sc
        kth = sorted(scores.values())[keep - 1]
        moves_p = mv[p * M:(p + 1) * M].cpu().numpy().tolist()
        for j in range(keep):
            k = moves_p.index(kept[p, j].tolist())
            assert scores[k] <= kth + 1e-3 * max(1.0, abs(kth)), (p, j, scores[k], kth)
    # screened steps: exact costs and occupancy after every applied move
    search.run_search(wh, lay, prob, costs, mixed, 4, M, 8, 0, sg=sg, keep=keep)
    cur_maps = prob.slot_map.cpu().numpy().reshape(inst.n_plans, -1)
    cur = wh_gen.Instance(inst.layout, inst.n_sku, inst.order_off, inst.line_sku, cur_maps.ravel(),
                          inst.plan_tour_off, prob.tour_off.cpu().numpy(), prob.order_seq.cpu().numpy())
    want = oracle.eval_plans(cur, slot_map=cur_maps.ravel(), slot_map_stride=inst.n_sku)
    assert np.array_equal(costs.plan_rr[:inst.n_plans].cpu().numpy(), want[3])
    words = (inst.layout.n_loc + 31) // 32
    bits = np.zeros((inst.n_plans, words), np.uint32)
    for p in range(inst.n_plans):
        for loc in cur_maps[p]:
            bits[p, loc >> 5] |= np.uint32(1 << (int(loc) & 31))
    assert np.array_equal(prob.loc_used.cpu().numpy().view(np.uint32).reshape(inst.n_plans, words), bits)
    assert lay.status() == 0
    sg.close()
    lay.close()


def test_trained_prescreen_beats_keeping_without_it(gpu_lib):
    """What the trained network gains: three screened searches from the same
    paper-scale start over the same move sets, each scoring exactly 4 of the
    64 moves of every plan per step (equal exact re-scores), keeping the 4
    moves that (a) the trained network predicts best, (b) an untrained
    network of the same shape predicts best, (c) a seeded random draw picks.
    The trained prescreen lowers the plans' total optimal cost the most."""
    import torch
    wh = gpu_lib
    n, M, keep, steps = 256, 64, search.keep_count(64), 12
    # training data: the exact optimal lengths of tours of other plans of the
    # same generator
    tr_inst = wh_gen.paperscale(seed=4, n_plans=2048, plan_base=1 << 20)
    lay_t = wh.Layout.of(tr_inst.layout)
    tr_prob = wh.to_device(tr_inst)
    X, t = search.training_set(wh, lay_t, tr_prob, wh.evaluate(lay_t, tr_prob), tr_inst.layout)
    trained = wh.Surrogate(31)
    search.train(trained, X, t, 400, 4096, 2e-3)
    untrained = wh.Surrogate(32)
    lay_t.close()
    inst = wh_gen.paperscale(seed=5, n_plans=n)
    moves = [moves_for(inst, 33, s, M) for s in range(steps)]
    gen = torch.Generator(device="cuda").manual_seed(34)
    rand_idx = [torch.argsort(torch.rand((n, M), device="cuda", generator=gen), dim=1)[:, :keep] for _ in moves]

    def run(arm):
        lay, prob, costs = setup(wh, inst)
        start = int(costs.plan_rr[:n].sum().item())
        cache = search.new_cache(prob)
        for s, mv in enumerate(moves):
            if arm == "random":
                kept = mv.view(n, M, 4)[torch.arange(n, device="cuda")[:, None], rand_idx[s]].reshape(-1, 4)
                lay.ls_step(prob, costs, kept.contiguous(), keep, 24)
            else:
                sg = trained if arm == "trained" else untrained
                search.screened_step(lay, sg, prob, costs, mv, M, keep, 24, 0, cache)
        end = int(costs.plan_rr[:n].sum().item())
        assert lay.status() == 0
        lay.close()
        return start - end

    gain = {arm: run(arm) for arm in ("trained", "untrained", "random")}
    assert gain["trained"] > 0
    assert gain["trained"] > gain["random"] and gain["trained"] > gain["untrained"], gain
    trained.close()
    untrained.close()
