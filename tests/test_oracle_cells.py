"""Pins of the oracle's cell division (cell edge = cutoff, rebuilt every step;
section "Design concept of CAMUS") and of the periodic wrap (Fig. 1,
boundary check): geometric invariants and tie cases."""
import numpy as np
import pytest

import oracle as O


def _sys(L, n):
    return O.System(L, np.zeros(n, np.int32), [[25.0]], 4.5, 1.0, 0.04)


@pytest.mark.parametrize("L", [(10.0, 10.0, 10.0), (8.37, 13.2, 23.99), (3.0, 3.0, 3.0)])
def test_cell_keys_locate_each_bead_in_its_cell(L):
    L = np.array(L)
    rng = np.random.default_rng(1)
    n = 5000
    pos = rng.uniform(0, 1, (n, 3)) * L
    s = _sys(L, n)
    nc, inv_h = O.cell_dims(s)
    assert np.all(nc == np.floor(L)) and np.all(L / nc >= 1.0)
    key = O.cell_keys(s, pos).astype(np.int64)
    assert key.min() >= 0 and key.max() < np.prod(nc)
    c = np.stack([key % nc[0], (key // nc[0]) % nc[1], key // (nc[0] * nc[1])], axis=1)
    h = L / nc
    lo, hi = c * h, (c + 1) * h
    tol = 1e-12 * L
    assert np.all(pos >= lo - tol) and np.all(pos <= hi + tol)


def test_cell_key_tie_cases():
    L = 10.0
    pos = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 5.0], [np.nextafter(10.0, 0), 9.5, 0.5],
                    [np.nextafter(3.0, 0), np.nextafter(4.0, 10), 9.999999999999]])
    s = _sys(L, 4)
    k = O.cell_keys(s, pos)
    assert k[0] == 0
    assert k[1] == (5 * 10 + 4) * 10 + 3          # exactly on faces: the upper cell
    assert k[2] == (0 * 10 + 9) * 10 + 9          # L - eps clamps into the last cell
    assert k[3] == (9 * 10 + 4) * 10 + 2
    # non-integer box: h = L / floor(L) > 1
    s2 = _sys(12.5, 1)
    nc, inv_h = O.cell_dims(s2)
    assert nc[0] == 12 and inv_h[0] == 12 / 12.5
    assert O.cell_keys(s2, np.array([[12.5 / 12 * 5, 0, 0]]))[0] in (4, 5)


def test_cell_sort_is_canonical():
    rng = np.random.default_rng(2)
    L = np.array([9.0, 7.5, 6.2])
    n = 4000
    pos = rng.uniform(0, 1, (n, 3)) * L
    s = _sys(L, n)
    key = O.cell_keys(s, pos)
    order, start = O.cell_sort(s, key)
    nc, _ = O.cell_dims(s)
    assert sorted(order.tolist()) == list(range(n))            # a bijection
    ks = key[order].astype(np.int64)
    assert np.all(np.diff(ks) >= 0)                            # cells non-decreasing
    same = np.diff(ks) == 0
    assert np.all(np.diff(order)[same] > 0)                    # ids ascending inside a cell
    counts = np.bincount(key.astype(np.int64), minlength=int(np.prod(nc)))
    assert np.array_equal(np.diff(start), counts)
    assert start[0] == 0 and start[-1] == n
    for c in rng.integers(0, np.prod(nc), 50):
        assert np.all(key[order[start[c]:start[c + 1]]] == c)


def test_wrap_into_box():
    L = np.array([10.0, 7.3, 3.0])
    rng = np.random.default_rng(4)
    x = rng.uniform(-25, 25, (3000, 3))
    x[:5] = [[10.0, 7.3, 3.0], [-1e-300, -0.0, 0.0], [-1e-17, 7.3 - 1e-16, 6.0],
             [20.0, 14.6, -3.0], [np.nextafter(10.0, 11), 0, 0]]
    s = _sys(L, x.shape[0])
    y = O.wrap(s, x)
    assert np.all(y >= 0.0) and np.all(y < L)
    k = (x - y) / L
    assert np.allclose(k, np.round(k), atol=1e-12)
    assert np.all(y[0] == 0.0)
    assert np.all(y[3] == 0.0)


def test_wrap_just_below_multiples_of_the_box():
    # x one ulp below k*L: x/L can round up to k, so x - L*floor(x/L) is a tiny
    # negative number that must still land inside [0, L)
    for Lx in (7.3, 10.0, 12.7, 3.3, 23.99):
        xs = []
        for k in range(-6, 7):
            for t in range(1, 4):
                x = k * Lx
                for _ in range(t):
                    x = np.nextafter(x, -np.inf)
                xs.append(x)
                xs.append(np.nextafter(k * Lx, np.inf))
        x = np.array(xs)
        pos = np.stack([x, np.full_like(x, 0.5), np.full_like(x, 0.5)], axis=1)
        s = _sys((Lx, 5.0, 5.0), x.size)
        y = O.wrap(s, pos)[:, 0]
        assert np.all(y >= 0.0) and np.all(y < Lx)

