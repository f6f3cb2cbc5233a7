"""Seeded synthetic catalogues generated on the GPU, for the full-size
workloads (hundreds of millions of sources) that the host generator in
``synth`` would take minutes to draw.

The same recipes as ``synth`` (uniform on the sphere, latitude density
profiles by rejection on sin(latitude), spherical caps, Gaussian offsets
moved along great circles, unique ids), drawn with torch's counter-based
Philox generator on the device. Like ``synth`` this module holds no
cross-match arithmetic, and both sides consume what it draws: the CUDA
library reads the device tensors, the oracle a host copy of a sample.

Positions are degrees (float64); sizes arcsec; angles degrees. ``frame`` is
0 (equatorial) or 1 (galactic).
"""

from __future__ import annotations

import math

import numpy as np
import torch

ARCSEC = math.pi / 648000.0
EQ, GAL = 0, 1
CIRCLE, ELLIPSE, RECT = 0, 1, 2
JOIN_NAMES = ("and", "or", "all1", "all2", "not1_2", "not2_1", "xor")


def generator(seed: int, device="cuda") -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


def _u(g, n, lo, hi):
    return torch.rand(n, generator=g, device=g.device, dtype=torch.float64) * (hi - lo) + lo


def uniform_box(g, n, lon_lo, lon_hi, lat_lo, lat_hi):
    """Uniform per solid angle on lon in [lon_lo, lon_hi), sin(lat) uniform."""
    lon = torch.remainder(_u(g, n, lon_lo, lon_hi), 360.0)
    s = _u(g, n, math.sin(math.radians(lat_lo)), math.sin(math.radians(lat_hi)))
    return lon, torch.rad2deg(torch.asin(s))


def latitude_profile(g, n, density, lat_max_deg=90.0, lon_lo=0.0, lon_hi=360.0,
                     chunk=1 << 27):
    """n positions with surface density proportional to density(|lat| deg)
    (a torch function, values <= 1), by rejection on sin(lat)."""
    smax = math.sin(math.radians(lat_max_deg))
    out_lon, out_lat, have = [], [], 0
    while have < n:
        m = min(chunk, max(1 << 16, int(1.2 * (n - have) / 0.2)))
        lat = torch.rad2deg(torch.asin(_u(g, m, -smax, smax)))
        keep = _u(g, m, 0.0, 1.0) < density(lat.abs())
        lat = lat[keep]
        lon = torch.remainder(_u(g, lat.numel(), lon_lo, lon_hi), 360.0)
        out_lon.append(lon)
        out_lat.append(lat)
        have += lat.numel()
    return torch.cat(out_lon)[:n].contiguous(), torch.cat(out_lat)[:n].contiguous()


def destination(lon, lat, dist_rad, bearing_rad):
    """The point at angular distance dist from (lon, lat) along the great
    circle leaving it at the given bearing (east of north)."""
    lr, br = torch.deg2rad(lon), torch.deg2rad(lat)
    cl, sl, cb, sb = torch.cos(lr), torch.sin(lr), torch.cos(br), torch.sin(br)
    st, ct = torch.sin(bearing_rad), torch.cos(bearing_rad)
    cd, sd = torch.cos(dist_rad), torch.sin(dist_rad)
    # unit vector p, east e = (-sl, cl, 0), north n = (-sb cl, -sb sl, cb)
    tx = -st * sl - ct * sb * cl
    ty = st * cl - ct * sb * sl
    tz = ct * cb
    qx = cd * cb * cl + sd * tx
    qy = cd * cb * sl + sd * ty
    qz = cd * sb + sd * tz
    lon2 = torch.remainder(torch.rad2deg(torch.atan2(qy, qx)), 360.0)
    lat2 = torch.rad2deg(torch.atan2(qz, torch.hypot(qx, qy)))
    return lon2, lat2


def gaussian_offsets(g, lon, lat, sigma_arcsec):
    """Copies of (lon, lat) moved by an isotropic Gaussian offset of width
    sigma (a scalar or a tensor); also returns the true offset in arcsec."""
    n = lon.numel()
    x = torch.randn(n, generator=g, device=g.device, dtype=torch.float64) * sigma_arcsec
    y = torch.randn(n, generator=g, device=g.device, dtype=torch.float64) * sigma_arcsec
    rho = torch.hypot(x, y)
    lon2, lat2 = destination(lon, lat, rho * ARCSEC, torch.atan2(x, y))
    return lon2, lat2, rho


def cap(g, n, lon0, lat0, radius_deg):
    """Uniform per solid angle inside the spherical cap of the given radius."""
    c = _u(g, n, math.cos(math.radians(radius_deg)), 1.0)
    full = lambda v: torch.full((n,), float(v), dtype=torch.float64, device=g.device)  # noqa: E731
    return destination(full(lon0), full(lat0), torch.acos(c), _u(g, n, 0.0, 2 * math.pi))


def unique_ids(n, seed, device="cuda"):
    """n distinct positive int64 ids: an odd multiplier is a bijection mod 2^63
    (the same ids as the host generator gives)."""
    rows = torch.arange(n, dtype=torch.int64, device=device) + (seed * 7919 + 1)
    mult = 0x9E3779B97F4A7C15 - (1 << 64)  # the same 64-bit pattern, as int64
    return (rows * mult) & ((1 << 63) - 1)


def _permute(g, n):
    return torch.randperm(n, generator=g, device=g.device)


def c3_profile(b):
    return (1.0 + 9.0 * torch.exp(-b / 10.0)) / 10.0


def c3(seed=1003, scale=1.0, special=10_000, device="cuda"):
    """All-sky circle cross-match, full size by default: surface density
    ~ 1 + 9 exp(-|b|/10 deg) in galactic latitude for both catalogues
    (given in galactic coordinates); A = 5e7 * scale, 60 % with a B
    counterpart offset by sigma = 0.5 arcsec; B = 2e8 * scale; r = 2 arcsec;
    int64 ids. ``special`` A within 0.5 deg of each pole and ``special``
    across longitude 0/360, all with counterparts. Device tensors."""
    g = generator(seed, device)
    n_a, n_b = int(round(50_000_000 * scale)), int(round(200_000_000 * scale))
    special = min(special, n_a // 10)
    n_gen = n_a - 3 * special
    a_lon, a_lat = latitude_profile(g, n_gen, c3_profile)
    np_lon, np_lat = cap(g, special, 0.0, 90.0, 0.5)
    sp_lon, sp_lat = cap(g, special, 0.0, -90.0, 0.5)
    se_lon, se_lat = uniform_box(g, special, -0.5, 0.5, -60.0, 60.0)
    a_lon = torch.cat([a_lon, np_lon, sp_lon, se_lon])
    a_lat = torch.cat([a_lat, np_lat, sp_lat, se_lat])
    perm_a = _permute(g, n_a)
    a_lon, a_lat = a_lon[perm_a].contiguous(), a_lat[perm_a].contiguous()
    is_special = perm_a >= n_gen
    cand = torch.nonzero(~is_special).flatten()
    n_cp = int(round(0.6 * n_gen))
    pick = cand[_permute(g, cand.numel())[:n_cp]]
    src = torch.sort(torch.cat([pick, torch.nonzero(is_special).flatten()])).values
    cp_lon, cp_lat, rho = gaussian_offsets(g, a_lon[src], a_lat[src], 0.5)
    n_fresh = max(0, n_b - src.numel())
    fr_lon, fr_lat = latitude_profile(g, n_fresh, c3_profile)
    b_lon, b_lat = torch.cat([cp_lon, fr_lon]), torch.cat([cp_lat, fr_lat])
    perm_b = _permute(g, b_lon.numel())
    b_lon, b_lat = b_lon[perm_b].contiguous(), b_lat[perm_b].contiguous()
    inv = torch.empty_like(perm_b)
    inv[perm_b] = torch.arange(perm_b.numel(), device=device)
    return dict(name="c3", a_lon=a_lon, a_lat=a_lat, b_lon=b_lon, b_lat=b_lat,
                a_frame=GAL, b_frame=GAL, a_id=unique_ids(n_a, seed, device),
                b_id=unique_ids(b_lon.numel(), seed + 1, device),
                region=dict(shape=CIRCLE, a=2.0),
                truth=dict(a_row=src, b_row=inv[:src.numel()], rho_arcsec=rho))


def c5_catalogue(seed=1005, n_b=300_000_000, device="cuda"):
    """The resident B of the serving workload: n_b sources with C3's
    latitude profile, galactic coordinates, int64 ids. Device tensors."""
    g = generator(seed, device)
    b_lon, b_lat = latitude_profile(g, n_b, c3_profile)
    return dict(b_lon=b_lon, b_lat=b_lat, b_frame=GAL, b_id=unique_ids(n_b, seed + 1, device))


def c5_requests(b, seed=1006, n_pool=256, a_lo=1_000, a_hi=10_000_000, device="cuda"):
    """A pool of serving requests over B (``c5_catalogue``): each over a
    spherical cap with centre uniform on the sphere and diameter log-uniform
    in [0.1, 10] deg, n_A log-uniform in [a_lo, a_hi]; region shape uniform
    over circle / ellipse / rectangle, size log-uniform 0.5-30 arcsec, axis
    ratio 0.3-1, PA 0-180 deg, fixed or per-source (even odds); selection
    and join uniform over the 14 (all, best) x 7 combinations; input frame
    galactic or equatorial (even odds). A galactic request takes half its A
    as offset copies (sigma = 0.3 x size) of B sources inside its cap, half
    uniform in the cap; an equatorial request is uniform in a cap given in
    equatorial coordinates (its sources meet B wherever the cap falls).
    Device tensors; sizes are drawn on the host from the same seed. Each
    request records its cap (centre and radius in its own frame, degrees),
    the sigma of its offset copies and its largest region size (arcsec), so
    tests can cut B around it."""
    g = generator(seed, device)
    h = np.random.Generator(np.random.Philox(key=seed))
    bx = torch.cos(torch.deg2rad(b["b_lat"])) * torch.cos(torch.deg2rad(b["b_lon"]))
    by = torch.cos(torch.deg2rad(b["b_lat"])) * torch.sin(torch.deg2rad(b["b_lon"]))
    bz = torch.sin(torch.deg2rad(b["b_lat"]))
    out = []
    for _ in range(n_pool):
        c_lon = h.uniform(0.0, 360.0)
        c_lat = float(np.degrees(np.arcsin(h.uniform(-1.0, 1.0))))
        rad = 0.5 * float(np.exp(h.uniform(np.log(0.1), np.log(10.0))))
        n_a = int(np.exp(h.uniform(np.log(a_lo), np.log(a_hi))))
        shape = int(h.integers(0, 3))
        size = float(np.exp(h.uniform(np.log(0.5), np.log(30.0))))
        ratio = float(h.uniform(0.3, 1.0))
        per_source = bool(h.integers(0, 2))
        combo = int(h.integers(0, 14))
        frame = int(h.integers(0, 2))
        n_half = n_a // 2 if frame == GAL else 0
        u_lon, u_lat = cap(g, n_a - n_half, c_lon, c_lat, rad)
        if n_half:
            cl, cb = math.radians(c_lon), math.radians(c_lat)
            inside = torch.nonzero(bx * (math.cos(cb) * math.cos(cl)) + by * (math.cos(cb) * math.sin(cl))
                                   + bz * math.sin(cb) >= math.cos(math.radians(rad))).flatten()
            if inside.numel():
                pick = inside[torch.randint(0, inside.numel(), (n_half,), generator=g, device=device)]
                o_lon, o_lat, _ = gaussian_offsets(g, b["b_lon"][pick], b["b_lat"][pick], 0.3 * size)
            else:
                o_lon, o_lat = cap(g, n_half, c_lon, c_lat, rad)
            u_lon, u_lat = torch.cat([u_lon, o_lon]), torch.cat([u_lat, o_lat])
        region = dict(shape=shape)
        if per_source:
            a_col = torch.exp(_u(g, n_a, math.log(0.5), math.log(30.0)))
            region.update(a_col=a_col, b_col=a_col * _u(g, n_a, 0.3, 1.0),
                          pa_col=_u(g, n_a, 0.0, 180.0))
        else:
            region.update(a=size, b=size * ratio, pa=float(h.uniform(0.0, 180.0)))
        out.append(dict(lon=u_lon.contiguous(), lat=u_lat.contiguous(), frame=frame,
                        region=region, selection=3, join=JOIN_NAMES[combo % 7],
                        join_selection=1 if combo < 7 else 2,
                        cap=(c_lon, c_lat, rad), offset_sigma=0.3 * size if n_half else 0.0,
                        max_size=30.0 if per_source else size))
    return out


def poisson_arrivals(rate_per_s, duration_s, seed=1007):
    """Arrival times (s) of a Poisson stream, and the pool index of each."""
    h = np.random.Generator(np.random.Philox(key=seed))
    t, times = 0.0, []
    while True:
        t += h.exponential(1.0 / rate_per_s)
        if t >= duration_s:
            break
        times.append(t)
    return np.array(times), h


def c4(seed=1004, n_b=100_000_000, n_req=4096, a_lo=100, a_hi=1_000_000, device="cuda"):
    """Batched jobs, full size by default: B = n_b uniform on the whole sky
    (equatorial); n_req requests, each over a spherical cap with centre
    uniform on the sphere and diameter log-uniform in [0.1, 10] deg, n_A
    log-uniform in [a_lo, a_hi], half uniform in the cap and half offset
    copies (sigma = 0.3 x region size) of B sources drawn with replacement
    from the cap; shape uniform over circle / ellipse / rectangle, size
    log-uniform 0.5-30 arcsec, axis ratio 0.3-1, PA 0-180 deg, fixed or
    per-source (even odds); selection and join uniform over the 14
    (all, best) x 7 combinations. Device tensors; request parameters are
    drawn on the host from the same seed. Each request also records its cap
    (centre, radius) so tests can cut B around it."""
    g = generator(seed, device)
    h = np.random.Generator(np.random.Philox(key=seed))
    b_lon, b_lat = uniform_box(g, n_b, 0.0, 360.0, -90.0, 90.0)
    ub = torch.stack([torch.cos(torch.deg2rad(b_lat)) * torch.cos(torch.deg2rad(b_lon)),
                      torch.cos(torch.deg2rad(b_lat)) * torch.sin(torch.deg2rad(b_lon)),
                      torch.sin(torch.deg2rad(b_lat))])
    requests = []
    for _ in range(n_req):
        c_lon = h.uniform(0.0, 360.0)
        c_lat = float(np.degrees(np.arcsin(h.uniform(-1.0, 1.0))))
        rad = 0.5 * float(np.exp(h.uniform(np.log(0.1), np.log(10.0))))
        n_a = int(np.exp(h.uniform(np.log(a_lo), np.log(a_hi))))
        shape = int(h.integers(0, 3))
        size = float(np.exp(h.uniform(np.log(0.5), np.log(30.0))))
        ratio = float(h.uniform(0.3, 1.0))
        per_source = bool(h.integers(0, 2))
        combo = int(h.integers(0, 14))
        n_half = n_a // 2
        u_lon, u_lat = cap(g, n_a - n_half, c_lon, c_lat, rad)
        cl, cb = math.radians(c_lon), math.radians(c_lat)
        cvec = torch.tensor([math.cos(cb) * math.cos(cl), math.cos(cb) * math.sin(cl), math.sin(cb)],
                            dtype=torch.float64, device=device)
        inside = torch.nonzero(cvec @ ub >= math.cos(math.radians(rad))).flatten()
        if inside.numel() and n_half:
            pick = inside[torch.randint(0, inside.numel(), (n_half,), generator=g, device=device)]
            o_lon, o_lat, _ = gaussian_offsets(g, b_lon[pick], b_lat[pick], 0.3 * size)
        else:
            o_lon, o_lat = cap(g, n_half, c_lon, c_lat, rad)
        region = dict(shape=shape)
        if per_source:
            a_col = torch.exp(_u(g, n_a, math.log(0.5), math.log(30.0)))
            region.update(a_col=a_col, b_col=a_col * _u(g, n_a, 0.3, 1.0),
                          pa_col=_u(g, n_a, 0.0, 180.0))
        else:
            region.update(a=size, b=size * ratio, pa=float(h.uniform(0.0, 180.0)))
        requests.append(dict(lon=torch.cat([u_lon, o_lon]).contiguous(),
                             lat=torch.cat([u_lat, o_lat]).contiguous(), region=region,
                             selection=3, join=JOIN_NAMES[combo % 7],
                             join_selection=1 if combo < 7 else 2,
                             cap=(c_lon, c_lat, rad), offset_sigma=0.3 * size,
                             max_size=30.0 if per_source else size))
    return dict(name="c4", b_lon=b_lon, b_lat=b_lat, b_frame=EQ, requests=requests)


def values(seed=1008, n_a=50_000_000, n_b=200_000_000, device="cuda"):
    """Exact Value case (paper §2.1): int64 key columns. B holds n_b keys: 90 %
    distinct ids and 10 % repeats of them (so some keys appear twice or more);
    A holds n_a keys, 60 % drawn from B's keys (with replacement), 40 %
    fresh ids that match nothing. Device tensors."""
    g = generator(seed, device)
    n_distinct = int(n_b * 0.9)
    ids = unique_ids(n_distinct + n_a, seed, device)
    b_ids = ids[:n_distinct]
    rep = b_ids[torch.randint(0, n_distinct, (n_b - n_distinct,), generator=g, device=device)]
    b = torch.cat([b_ids, rep])[_permute(g, n_b)].contiguous()
    n_hit = int(n_a * 0.6)
    hit = b[torch.randint(0, n_b, (n_hit,), generator=g, device=device)]
    fresh = ids[n_distinct:n_distinct + (n_a - n_hit)]
    a = torch.cat([hit, fresh])[_permute(g, n_a)].contiguous()
    return dict(a_keys=a, b_keys=b)
