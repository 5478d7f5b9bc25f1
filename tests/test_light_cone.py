"""The light-cone sampling that checks the GPU path against the oracle at
full lattice sizes: the oracle's values after k steps at sampled cells,
each computed on the (2k + 1)^3 neighbourhood of the cell alone, equal the
values of the oracle run on the whole periodic lattice bit for bit (corner
cells included, whose neighbourhoods wrap across every face); one step more
than the neighbourhood allows does change them.  CPU."""
import numpy as np

import oracle
import workloads as W
from tests._helpers import light_cone_cells, light_cone_oracle


def test_light_cone_values_equal_the_whole_lattice():
    k = 4
    w = W.random_box(L=24, steps=k, sigma=3.0)
    p = oracle.Params(**w.params())
    st = oracle.init(p, w.n, w.eps, w.beta)
    oracle.run(p, st, k)
    n, e, b, _ = oracle.macro(p, st)
    cells = light_cone_cells(w, 20, seed=7)
    ln, le, lb = light_cone_oracle(w, k, cells)
    zs, ys, xs = (np.array(c) for c in zip(*cells))
    assert np.array_equal(ln, n[zs, ys, xs])
    assert np.array_equal(le, e[zs, ys, xs])
    assert np.array_equal(lb, b[:, zs, ys, xs])
    # the neighbourhood is no larger than needed: k + 1 steps on it differ
    p_sub = oracle.Params(**{**w.params(), "nx": 2 * k + 1, "ny": 2 * k + 1, "nz": 2 * k + 1})
    r = np.arange(-k, k + 1)
    z, y, x = cells[-1]
    iz, iy, ix = (z + r) % w.nz, (y + r) % w.ny, (x + r) % w.nx
    sub = lambda a: np.ascontiguousarray(a[..., iz[:, None, None], iy[None, :, None], ix[None, None, :]])
    s2 = oracle.init(p_sub, sub(w.n), sub(w.eps), sub(w.beta))
    oracle.run(p_sub, s2, k + 1)
    full = oracle.init(p, w.n, w.eps, w.beta)
    oracle.run(p, full, k + 1)
    assert oracle.macro(p_sub, s2)[1][k, k, k] != oracle.macro(p, full)[1][z, y, x]
