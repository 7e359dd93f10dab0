"""How mf_advance_batch arranges films into launches (host logic of the C library, no GPU)."""
import math
import os

import numpy as np

import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CORESIDENT = 304          # 2 CTAs on each of 152 SMs


@pytest.fixture(scope="module")
def plan():
    from paper_1801_04869_gb300 import build, native
    if not os.path.exists(native.LIB_PATH):
        build.build()
    return native.batch_plan


def cost(g):
    c = g[0] * g[1]
    return c * math.log2(c)


def own_grid(g):
    # the size rule of a film's own launch: one CTA per column item, at most the co-resident CTAs
    return min(CORESIDENT, g[0] // 2 + 1)


def check(films, own, nl, order, launch, ctas, coresident=CORESIDENT, work=None):
    n = len(films)
    w = work if work is not None else [cost(f) for f in films]
    assert sorted(order) == list(range(n))
    costs = [w[i] for i in order]
    assert all(a >= b for a, b in zip(costs, costs[1:]))
    shared = [i for i in order if launch[i] >= 0]
    assert [launch[i] for i in shared] == sorted(launch[i] for i in shared)
    assert set(launch[i] for i in shared) == set(range(nl))
    for i in range(n):
        if own[i] >= coresident:
            assert launch[i] == -1 and ctas[i] == coresident
        else:
            assert launch[i] >= 0 and 1 <= ctas[i] <= own[i]
    for j in range(nl):
        m = [i for i in shared if launch[i] == j]
        assert 1 <= len(m) <= min(256, coresident)
        assert sum(ctas[i] for i in m) <= coresident
        c = [w[i] for i in m]
        # every film's share of the grid in proportion to its work is at least one CTA
        assert sum(c) <= coresident * min(c) * (1 + 1e-12)
        # the next launch's first film would have broken that (unless the 256-film cap closed it)
        nxt = [i for i in shared if launch[i] == j + 1]
        if nxt and len(m) < min(256, coresident):
            cn = w[nxt[0]]
            assert sum(c) + cn > coresident * cn
        # no CTA can move between two films of the launch and lower its largest work per CTA
        # (with the grid full or every film at its own launch width)
        worst = max(m, key=lambda i: w[i] / ctas[i])
        wr = w[worst] / ctas[worst]
        if ctas[worst] < own[worst]:
            assert sum(ctas[i] for i in m) == coresident
            for a in m:
                if a != worst and ctas[a] > 1:
                    assert w[a] / (ctas[a] - 1) >= wr * (1 - 1e-12)


def test_sweep_of_256_films(plan):
    wls = W.film_batch(256, seed=3, max_side=512, precision=1)
    films = [(wl.nx, wl.ny) for wl in wls]
    own = [own_grid(f) for f in films]
    nl, order, launch, ctas = plan([f[0] for f in films], [f[1] for f in films], own, CORESIDENT)
    check(films, own, nl, order, launch, ctas)
    big = [i for i, f in enumerate(films) if f[0] == 1024]
    assert big and all(launch[i] == -1 for i in big)
    # 512^2 films share one launch, 256^2 films the next
    assert len({launch[i] for i, f in enumerate(films) if f[0] == 512}) == 1
    assert len({launch[i] for i, f in enumerate(films) if f[0] == 256}) == 1
    assert nl == 2


def test_edge_cases(plan):
    assert plan([], [], [], CORESIDENT)[0] == 0
    nl, order, launch, ctas = plan([128], [128], [65], CORESIDENT)
    assert (nl, launch, ctas) == (1, [0], [65])
    nl, order, launch, ctas = plan([2048, 2048], [2048, 2048], [304, 304], CORESIDENT)
    assert (nl, launch) == (0, [-1, -1])
    # 300 equal small films: the 256-film cap splits them
    films = [(128, 128)] * 300
    own = [65] * 300
    nl, order, launch, ctas = plan([128] * 300, [128] * 300, own, CORESIDENT)
    check(films, own, nl, order, launch, ctas)
    assert nl == 2 and sum(1 for x in launch if x == 0) == 256
    assert order == list(range(300))          # equal films keep their order
    # uneven films, one GPU's worth of CTAs fewer than films would need at their own widths
    films = [(256, 256)] * 3 + [(128, 64)] * 50 + [(512, 256)] * 2
    own = [own_grid(f) for f in films]
    nl, order, launch, ctas = plan([f[0] for f in films], [f[1] for f in films], own, 96)
    check(films, own, nl, order, launch, ctas, coresident=96)
    with pytest.raises(ValueError):
        plan([128], [128], [0], CORESIDENT)
    with pytest.raises(ValueError):
        plan([128], [128], [65], 0)


def test_measured_work_weights(plan):
    """Equal grids, unequal measured work: the film that needed the most outside iterations
    gets the most CTAs, and the largest work per CTA is as small as whole CTAs allow."""
    films = [(256, 256)] * 40
    own = [own_grid(f) for f in films]
    r = np.random.default_rng(5)
    work = [cost(f) * (19 * 3.5 + 14 * 3.5 * it) for f, it in zip(films, r.uniform(2, 40, 40))]
    nl, order, launch, ctas = plan([256] * 40, [256] * 40, own, CORESIDENT, work=work)
    check(films, own, nl, order, launch, ctas, work=work)
    assert nl == 1 and sum(ctas) == CORESIDENT
    heavy = max(range(40), key=lambda i: work[i])
    assert ctas[heavy] == max(ctas) and order[0] == heavy
    with pytest.raises(ValueError):
        plan([128], [128], [65], CORESIDENT, work=[0.0])
