"""Host-side planning of a batch (no GPU): size classes and the tile lists of the
grouped tensor-core launches, through the library's host-only entry point."""
import numpy as np
import pytest

from paper_2304_02327_gb300 import api, workloads as wl


@pytest.fixture(scope="module")
def lib():
    from paper_2304_02327_gb300 import build
    build.build()
    return api.lib()


def expected_tiles(n1, n2, nc_cap, mode):
    """Every (instance, row tile, column split) a direction needs: rows of 128
    fibres, output columns in the fewest splits of width <= nc_cap (multiple of 16)."""
    out = set()
    for j, (a, b) in enumerate(zip(n1, n2)):
        k, rows = (a, b) if mode == 1 else (b, a)
        n16 = -(-k // 16) * 16
        sp = -(-n16 // nc_cap)
        nc = -(-(-(-n16 // sp)) // 16) * 16
        sp = -(-n16 // nc)
        for r in range(-(-rows // 128)):
            for s in range(sp):
                out.add((j, r, s))
    return out


@pytest.mark.parametrize("nc_cap", [160, 128, 96, 64, 16])
@pytest.mark.parametrize("mode", [1, 2])
def test_tile_plan_covers_every_tile_once(lib, nc_cap, mode):
    probs = wl.batched_allen_cahn(count=40, seed=4)
    n1 = [p.n[0] for p in probs]
    n2 = [p.n[0] + (7 if j % 3 == 0 else 0) for j, p in enumerate(probs)]   # some n1 != n2
    t = api.batch_tile_plan(n1, n2, "bf16x3", nc_cap, mode)
    got = [tuple(r[:3]) for r in t]
    assert len(got) == len(set(got))                                    # no tile twice
    assert set(got) == expected_tiles(n1, n2, nc_cap, mode)             # exact cover
    # one size class per distinct (n1, n2), consistent for all tiles of an instance
    cls = {}
    for inst, _, _, c in t:
        assert cls.setdefault(inst, c) == c
    keys = {}
    for inst, c in cls.items():
        assert keys.setdefault(c, (n1[inst], n2[inst])) == (n1[inst], n2[inst])
    assert len(keys) == len({(a, b) for a, b in zip(n1, n2)})


def test_tile_plan_orders_by_decreasing_cost(lib):
    """Tiles come largest first (cost ~ K-blocks x (256 + nc)), so the round-robin over
    the CTAs hands every CTA a similar share."""
    n = [48, 512, 96, 320, 512, 64]
    t = api.batch_tile_plan(n, n, "tf32x3", 128, 1)

    def cost(k):
        n16 = -(-k // 16) * 16
        sp = -(-n16 // 128)
        nc = -(-(-(-n16 // sp)) // 16) * 16
        return -(-k // 32) * (256 + nc)         # TF32: 32-value K-blocks

    c = [cost(n[i]) for i in t[:, 0]]
    assert all(a >= b for a, b in zip(c, c[1:]))
    assert n[t[0, 0]] == 512 and n[t[-1, 0]] == 48


def test_tile_plan_rejects_bad_requests(lib):
    with pytest.raises(api.PhisplitError):
        api.batch_tile_plan([64], [64], "bf16x3", 100, 1)          # not a multiple of 16
    with pytest.raises(api.PhisplitError):
        api.batch_tile_plan([64], [64], "fp64", 128, 1)            # mixed forms only
    sizes = list(range(16, 16 * 34, 16))                           # 33 size classes
    with pytest.raises(api.PhisplitError) as e:
        api.batch_tile_plan(sizes, sizes, "bf16x3", 128, 1)
    assert e.value.code == -3
