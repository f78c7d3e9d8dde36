"""The vertical cell lookup of the step kernels, emulated in FP32 with numpy: a table of
bins of the smallest level spacing / 1.2, each holding the cell 0.05 bin below its lower
edge, corrected by one comparison with the next level, gives the exact cell (last level
<= z, clamped to [0, nz-2]) for any z, including every level, every bin edge and their
neighbouring floats, on the realistic levels and on random irregular level sets."""
import numpy as np

import lpm_inputs as li


def _table(zf):
    nz = len(zf)
    min_sp = min(float(zf[k + 1]) - float(zf[k]) for k in range(nz - 1))
    span = float(zf[-1]) - float(zf[0])
    n = int(np.ceil(span / (min_sp / 1.2)) + 1)
    inv_h = np.float32((n - 1) / span)
    lut = np.empty(n, dtype=np.int64)
    for b in range(n):
        zb = float(zf[0]) + (b - 0.05) / float(inv_h)
        lut[b] = min(int(np.searchsorted(zf.astype(np.float64), zb, side="right")) - 1, nz - 2)
    return np.maximum(lut, 0), inv_h


def _lookup(zf, lut, inv_h, z):
    nz = len(zf)
    b = np.trunc(((z - zf[0]).astype(np.float32) * inv_h).astype(np.float32)).astype(np.int64)
    b = np.clip(b, 0, len(lut) - 1)
    k0 = lut[b]
    up = (k0 < nz - 2) & (z >= zf[np.minimum(k0 + 1, nz - 1)])
    return k0 + up


def _probe_points(zf, inv_h, n_lut, rng, n):
    lo, hi = float(zf[0]) - 10.0, float(zf[-1]) + 100.0
    edges = (float(zf[0]) + np.arange(n_lut) / float(inv_h)).astype(np.float32)
    pts = [rng.uniform(lo, hi, n).astype(np.float32), zf, edges]
    for p in (zf, edges):
        pts += [np.nextafter(p, np.float32(-1e9)), np.nextafter(p, np.float32(1e9))]
    return np.concatenate(pts).astype(np.float32)


def _check(zf, rng, n):
    lut, inv_h = _table(zf)
    z = _probe_points(zf, inv_h, len(lut), rng, n)
    exact = np.clip(np.searchsorted(zf, z, side="right") - 1, 0, len(zf) - 2)
    got = _lookup(zf, lut, inv_h, z)
    assert np.array_equal(got, exact)


def test_level_lookup_exact_on_realistic_levels():
    zf = np.asarray(li.make_cfg1(n_particles=1, n_steps=1).z_levels, dtype=np.float32)
    _check(zf, np.random.default_rng(0), 200_000)


def test_level_lookup_exact_on_random_levels():
    rng = np.random.default_rng(7)
    for _ in range(100):
        nz = int(rng.integers(2, 64))
        d = rng.uniform(0.5, 300.0, nz - 1) * rng.uniform(0.01, 1.0, nz - 1) ** rng.uniform(0, 3)
        z0 = 0.0 if rng.uniform() < 0.5 else rng.uniform(-50.0, 50.0)
        zf = np.concatenate([[z0], z0 + np.cumsum(d)]).astype(np.float32)
        if np.any(np.diff(zf) <= 0):
            continue
        if (zf[-1] - zf[0]) / (np.diff(zf).min() / 1.2) > 4096:
            continue
        _check(zf, rng, 5000)
