"""Seeded synthetic catalogues shaped like the paper's workloads.

The paper's own inputs (Hi-GAL clumps against UKIDSS/GLIMPSE compact
sources, §3, and the unnamed public catalogues of §4) are not available; these
generators stand in for them with the shapes, sizes and density structure of
the five benchmark workloads. They are the ONE module both the CUDA path and
the oracle consume, so they hold no cross-match arithmetic: they only draw
positions (uniform on the sphere, latitude density profiles by rejection on
sin(latitude), Gaussian offsets moved along great circles) and region
parameters. Every draw comes from numpy's counter-based Philox generator with
a fixed seed.

Positions are degrees (float64); sizes are arcsec; position angles are
degrees. ``frame`` is 0 (equatorial) or 1 (galactic).
"""

from __future__ import annotations

import numpy as np

ARCSEC = np.pi / 648000.0
EQ, GAL = 0, 1
CIRCLE, ELLIPSE, RECT = 0, 1, 2


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=seed))


def uniform_box(g, n, lon_lo, lon_hi, lat_lo, lat_hi):
    """Uniform per solid angle on lon in [lon_lo, lon_hi), sin(lat) uniform."""
    lon = g.uniform(lon_lo, lon_hi, n) % 360.0
    s = g.uniform(np.sin(np.radians(lat_lo)), np.sin(np.radians(lat_hi)), n)
    return lon, np.degrees(np.arcsin(s))


def latitude_profile(g, n, density, lat_max_deg=90.0, lon_lo=0.0, lon_hi=360.0,
                     chunk=1 << 24):
    """n positions with a surface density proportional to density(|lat| deg)
    (density <= 1), drawn by rejection on sin(lat)."""
    out_lon, out_lat, have = [], [], 0
    smax = np.sin(np.radians(lat_max_deg))
    while have < n:
        m = min(chunk, max(1024, int(1.2 * (n - have) / 0.2)))
        lat = np.degrees(np.arcsin(g.uniform(-smax, smax, m)))
        keep = g.uniform(0.0, 1.0, m) < density(np.abs(lat))
        lat = lat[keep]
        lon = g.uniform(lon_lo, lon_hi, lat.size) % 360.0
        out_lon.append(lon)
        out_lat.append(lat)
        have += lat.size
    return np.concatenate(out_lon)[:n], np.concatenate(out_lat)[:n]


def _unit(lon, lat):
    l, b = np.radians(lon), np.radians(lat)
    return np.stack([np.cos(b) * np.cos(l), np.cos(b) * np.sin(l), np.sin(b)])


def destination(lon, lat, dist_rad, bearing_rad):
    """The point at angular distance dist from (lon, lat) along the great
    circle leaving it at the given bearing (east of north)."""
    l, b = np.radians(lon), np.radians(lat)
    p = _unit(lon, lat)
    east = np.stack([-np.sin(l), np.cos(l), np.zeros_like(l)])
    north = np.stack([-np.sin(b) * np.cos(l), -np.sin(b) * np.sin(l), np.cos(b)])
    t = np.sin(bearing_rad) * east + np.cos(bearing_rad) * north
    q = np.cos(dist_rad) * p + np.sin(dist_rad) * t
    lon2 = np.degrees(np.arctan2(q[1], q[0])) % 360.0
    lat2 = np.degrees(np.arctan2(q[2], np.hypot(q[0], q[1])))
    return lon2, lat2


def gaussian_offsets(g, lon, lat, sigma_arcsec):
    """Copies of (lon, lat) moved by an isotropic Gaussian offset of width
    sigma; also returns the true offset in arcsec."""
    x = g.normal(0.0, sigma_arcsec, lon.size)
    y = g.normal(0.0, sigma_arcsec, lon.size)
    rho = np.hypot(x, y)
    lon2, lat2 = destination(lon, lat, rho * ARCSEC, np.arctan2(x, y))
    return lon2, lat2, rho


def cap(g, n, lon0, lat0, radius_deg):
    """Uniform per solid angle inside the spherical cap of the given radius."""
    c = g.uniform(np.cos(np.radians(radius_deg)), 1.0, n)
    return destination(np.full(n, lon0), np.full(n, lat0), np.arccos(c),
                       g.uniform(0.0, 2 * np.pi, n))


def unique_ids(n, seed):
    """n distinct positive int64 ids: an odd multiplier is a bijection mod 2^63."""
    rows = np.arange(n, dtype=np.uint64) + np.uint64(seed * 7919 + 1)
    ids = (rows * np.uint64(0x9E3779B97F4A7C15)) & np.uint64((1 << 63) - 1)
    return ids.astype(np.int64)


def _shuffle(g, *cols):
    perm = g.permutation(cols[0].size)
    return perm, [c[perm] for c in cols]


def c1(seed=1001):
    """Plain circle cross-match: A = 10,000 uniform on RA [150, 151] deg,
    Dec [2, 3] deg; B = shifted copies (sigma 0.3 arcsec) of a random 70 % of A
    plus 3,000 fresh uniform sources; circle r = 1 arcsec; equatorial."""
    g = rng(seed)
    n_a, n_pl, n_fresh = 10_000, 7_000, 3_000
    a_lon, a_lat = uniform_box(g, n_a, 150.0, 151.0, 2.0, 3.0)
    src = g.choice(n_a, n_pl, replace=False)
    pl_lon, pl_lat, rho = gaussian_offsets(g, a_lon[src], a_lat[src], 0.3)
    fr_lon, fr_lat = uniform_box(g, n_fresh, 150.0, 151.0, 2.0, 3.0)
    perm, (b_lon, b_lat) = _shuffle(g, np.concatenate([pl_lon, fr_lon]),
                                    np.concatenate([pl_lat, fr_lat]))
    inv = np.argsort(perm)
    return dict(name="c1", a_lon=a_lon, a_lat=a_lat, b_lon=b_lon, b_lat=b_lat,
                a_frame=EQ, b_frame=EQ,
                region=dict(shape=CIRCLE, a=1.0),
                truth=dict(a_row=src.astype(np.int64), b_row=inv[:n_pl].astype(np.int64),
                           rho_arcsec=rho))


def c2(seed=1002, scale=1.0):
    """Clump-vs-compact-source case (the paper's §3 use): galactic
    l in [0, 60*scale] deg, |b| <= 1 deg, surface density ~ exp(-|b|/0.3 deg)
    for both catalogues; A = 200,000*scale clumps with per-source ellipses
    (semi-major 5-60 arcsec log-uniform, axis ratio 0.3-1, PA 0-180 deg);
    B = 5,000,000*scale point sources."""
    g = rng(seed)
    n_a, n_b = int(round(200_000 * scale)), int(round(5_000_000 * scale))
    lon_hi = 60.0 * scale
    prof = lambda b: np.exp(-b / 0.3)  # noqa: E731
    a_lon, a_lat = latitude_profile(g, n_a, prof, 1.0, 0.0, lon_hi)
    b_lon, b_lat = latitude_profile(g, n_b, prof, 1.0, 0.0, lon_hi)
    semi = np.exp(g.uniform(np.log(5.0), np.log(60.0), n_a))
    ratio = g.uniform(0.3, 1.0, n_a)
    pa = g.uniform(0.0, 180.0, n_a)
    return dict(name="c2", a_lon=a_lon, a_lat=a_lat, b_lon=b_lon, b_lat=b_lat,
                a_frame=GAL, b_frame=GAL,
                region=dict(shape=ELLIPSE, a_col=semi, b_col=semi * ratio, pa_col=pa))


def c3(seed=1003, scale=1.0, special=10_000):
    """All-sky circle cross-match: surface density ~ 1 + 9 exp(-|b|/10 deg) in
    galactic latitude (both catalogues given in galactic coordinates);
    A = 50,000,000*scale, of which 60 % have a B counterpart offset by
    sigma = 0.5 arcsec; B = 200,000,000*scale; r = 2 arcsec; int64 ids. Among
    the A, ``special`` sources lie within 0.5 deg of each pole of the frame and
    ``special`` straddle longitude 0/360, all with counterparts."""
    g = rng(seed)
    n_a, n_b = int(round(50_000_000 * scale)), int(round(200_000_000 * scale))
    special = min(special, n_a // 10)
    prof = lambda b: (1.0 + 9.0 * np.exp(-b / 10.0)) / 10.0  # noqa: E731
    n_gen = n_a - 3 * special
    a_lon, a_lat = latitude_profile(g, n_gen, prof)
    np_lon, np_lat = cap(g, special, 0.0, 90.0, 0.5)
    sp_lon, sp_lat = cap(g, special, 0.0, -90.0, 0.5)
    seam_lon, seam_lat = uniform_box(g, special, -0.5, 0.5, -60.0, 60.0)
    a_lon = np.concatenate([a_lon, np_lon, sp_lon, seam_lon])
    a_lat = np.concatenate([a_lat, np_lat, sp_lat, seam_lat])
    perm_a, (a_lon, a_lat) = _shuffle(g, a_lon, a_lat)
    n_cp = int(round(0.6 * n_gen))
    is_special = perm_a >= n_gen
    cand = np.nonzero(~is_special)[0]
    src = np.concatenate([g.choice(cand, n_cp, replace=False), np.nonzero(is_special)[0]])
    src.sort()
    cp_lon, cp_lat, rho = gaussian_offsets(g, a_lon[src], a_lat[src], 0.5)
    n_fresh = max(0, n_b - src.size)
    fr_lon, fr_lat = latitude_profile(g, n_fresh, prof)
    perm_b, (b_lon, b_lat) = _shuffle(g, np.concatenate([cp_lon, fr_lon]),
                                      np.concatenate([cp_lat, fr_lat]))
    inv = np.argsort(perm_b)
    return dict(name="c3", a_lon=a_lon, a_lat=a_lat, b_lon=b_lon, b_lat=b_lat,
                a_frame=GAL, b_frame=GAL, a_id=unique_ids(n_a, seed),
                b_id=unique_ids(b_lon.size, seed + 1),
                region=dict(shape=CIRCLE, a=2.0),
                truth=dict(a_row=src.astype(np.int64), b_row=inv[:src.size].astype(np.int64),
                           rho_arcsec=rho))


JOIN_NAMES = ("and", "or", "all1", "all2", "not1_2", "not2_1", "xor")


def c4(seed=1004, n_b=100_000_000, n_req=4096, a_lo=100, a_hi=1_000_000):
    """Batched jobs: B uniform on the whole sky; n_req requests, each over a
    spherical cap centred uniformly on the sphere with a diameter log-uniform
    in [0.1, 10] deg, n_A log-uniform in [a_lo, a_hi]; half of each request's
    A uniform in the cap, half offset copies (sigma = 0.3 x region size) of B
    sources drawn with replacement from the cap. Region shape uniform over
    circle / ellipse / rectangle, size log-uniform 0.5-30 arcsec, axis ratio
    0.3-1, PA 0-180 deg, fixed or per-source (even odds); selection and join
    uniform over the 14 (all, best) x 7 join combinations.
    B rows are generated cell by cell (1-degree declination bands cut into
    near-square RA cells) so the generator can find the B rows of a cap; the
    row order is then shuffled."""
    g = rng(seed)
    b_lon, b_lat = uniform_box(g, n_b, 0.0, 360.0, -90.0, 90.0)
    band = np.clip(np.floor(b_lat + 90.0), 0, 179).astype(np.int64)
    nra = np.maximum(1, np.floor(360.0 * np.cos(np.radians(np.minimum(
        np.abs(np.arange(180) - 90.0), np.abs(np.arange(180) - 89.0))))).astype(np.int64))
    cell = band * 512 + np.minimum(np.floor(b_lon / 360.0 * nra[band]).astype(np.int64), nra[band] - 1)
    order = np.argsort(cell, kind="stable")
    cell_sorted = cell[order]
    p_b = _unit(b_lon, b_lat)
    requests = []
    for r in range(n_req):
        c_lon = g.uniform(0.0, 360.0)
        c_lat = float(np.degrees(np.arcsin(g.uniform(-1.0, 1.0))))
        rad = 0.5 * float(np.exp(g.uniform(np.log(0.1), np.log(10.0))))
        n_a = int(np.exp(g.uniform(np.log(a_lo), np.log(a_hi))))
        shape = int(g.integers(0, 3))
        size = float(np.exp(g.uniform(np.log(0.5), np.log(30.0))))
        ratio = float(g.uniform(0.3, 1.0))
        per_source = bool(g.integers(0, 2))
        combo = int(g.integers(0, 14))
        n_half = n_a // 2
        u_lon, u_lat = cap(g, n_a - n_half, c_lon, c_lat, rad)
        # B rows inside the cap, from the cells the cap touches
        lo_band = int(np.clip(np.floor(c_lat - rad + 90.0), 0, 179))
        hi_band = int(np.clip(np.floor(c_lat + rad + 90.0), 0, 179))
        idx = []
        for bd in range(lo_band, hi_band + 1):
            a0 = np.searchsorted(cell_sorted, bd * 512)
            a1 = np.searchsorted(cell_sorted, bd * 512 + 512)
            idx.append(order[a0:a1])
        idx = np.concatenate(idx) if idx else np.empty(0, np.int64)
        pc = _unit(np.array([c_lon]), np.array([c_lat]))[:, 0]
        inside = idx[(pc @ p_b[:, idx]) >= np.cos(np.radians(rad))] if idx.size else idx
        if inside.size and n_half:
            pick = inside[g.integers(0, inside.size, n_half)]
            o_lon, o_lat, _ = gaussian_offsets(g, b_lon[pick], b_lat[pick], 0.3 * size)
        else:
            o_lon, o_lat = cap(g, n_half, c_lon, c_lat, rad)
        a_lon = np.concatenate([u_lon, o_lon])
        a_lat = np.concatenate([u_lat, o_lat])
        region = dict(shape=shape)
        if per_source:
            a_col = np.exp(g.uniform(np.log(0.5), np.log(30.0), n_a))
            region.update(a_col=a_col, b_col=a_col * g.uniform(0.3, 1.0, n_a),
                          pa_col=g.uniform(0.0, 180.0, n_a))
        else:
            region.update(a=size, b=size * ratio, pa=float(g.uniform(0.0, 180.0)))
        requests.append(dict(lon=a_lon, lat=a_lat, region=region,
                             selection=3, join=JOIN_NAMES[combo % 7],
                             join_selection=1 if combo < 7 else 2))
    perm = g.permutation(n_b)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(n_b)
    return dict(name="c4", b_lon=b_lon[perm], b_lat=b_lat[perm], b_frame=EQ, requests=requests,
                b_row_of_generated=inv)
