"""CPU replay of the forward projector's depth-ordered march: which 128-byte
lines of the quad volume each warp load touches, counted for the whole warp
and per 16-lane half (a 128-bit warp load is served one half-warp at a time,
and each half costs one L1 wavefront per distinct line it touches).

The replay follows the kernel's organisation, not its arithmetic.  A warp
holds 32 rays: 32 / AG pixels of one detector row at AG neighbouring angles of
one memory layout and march direction.  It marches slabs of the layout's depth
axis whose width D is the smallest per-sample advance in the warp; a lane with
a sample inside the slab loads the 16-byte quad element of its cell in plane
s (the load of plane s + 1 has the same pattern, one plane further).  Samples
follow the midpoint rule over the ray's clip to the zero-padded support,
K = ceil(len / step).  Frame: source DSO (cos t, sin t, 0), detector centre
-(DSD - DSO) (cos t, sin t, 0), e_u = (-sin t, cos t, 0), e_v = (0, 0, 1); the
layout of an angle is y-fastest when |cos t| > |sin t|.

    python -m paper_1905_03748_gb300.march_replay --workload cgls_512 --warps 400 [--variants]
"""
import argparse
import json

import numpy as np

PAD = 2  # zero planes around the volume in the quad layouts
LINE = 128  # bytes
QUAD = 16  # bytes per quad element


def layout(t: float) -> int:
    return 1 if abs(np.cos(t)) > abs(np.sin(t)) else 0


def rays(geo: dict, t: float, pixels: np.ndarray, row: int):
    """First sample (padded index coordinates in the layout's (f, m, s) order),
    per-sample step and sample count of the rays through detector pixels
    `pixels` of row `row` at angle t."""
    nx, ny, nz = geo["n_voxel"]
    d = np.asarray(geo["d_voxel"], float)
    off = np.asarray(geo.get("off_origin", (0.0, 0.0, 0.0)), float)
    nu, nv = geo["n_det"]
    du, dv = geo["d_det"]
    ou, ov = geo.get("off_det", (0.0, 0.0))
    dso, dsd = geo["DSO"], geo["DSD"]
    c, s = np.cos(t), np.sin(t)
    src = np.array([dso * c, dso * s, 0.0])
    centre = np.array([-(dsd - dso) * c, -(dsd - dso) * s, 0.0])
    eu, ev = np.array([-s, c, 0.0]), np.array([0.0, 0.0, 1.0])
    u = (pixels - (nu - 1) / 2.0) * du + ou
    v = (row - (nv - 1) / 2.0) * dv + ov
    pix = centre[None] + u[:, None] * eu[None] + v * ev[None]
    n = np.array([nx, ny, nz], float)
    # index coordinates: voxel centres at 0 .. n-1, support [-1, n]
    a = (src - off) / d + (n - 1) / 2.0
    r = (pix - src[None]) / d[None]
    t0, t1 = np.zeros(len(pixels)), np.ones(len(pixels))
    with np.errstate(divide="ignore", invalid="ignore"):
        for k in range(3):
            ta, tb = (-1.0 - a[k]) / r[:, k], (n[k] - a[k]) / r[:, k]
            t0 = np.maximum(t0, np.minimum(ta, tb))
            t1 = np.minimum(t1, np.maximum(ta, tb))
    length = np.maximum(t1 - t0, 0.0) * np.linalg.norm(pix - src[None], axis=1)
    step = geo.get("accuracy", 0.5) * d.min()
    K = np.where(t1 > t0, np.maximum(1, np.ceil(length / step - 1e-9)), 0).astype(int)
    h = (t1 - t0) / np.maximum(K, 1)
    lay = layout(t)
    order = [1, 0, 2] if lay else [0, 1, 2]  # (f, m, s)
    x0 = (a[None] + (t0 + 0.5 * h)[:, None] * r)[:, order] + PAD
    dx = (h[:, None] * r)[:, order]
    return x0, dx, K, lay


def replay(geo: dict, angles: np.ndarray, ag: int = 2, order: str = "interleaved",
           n_warps: int = 400, seed: int = 0, tile=(8, 1), march: str = "slabs") -> dict:
    """Replay n_warps random warps; lines per load request, whole warp and
    summed over 16-lane halves, and lanes taking a sample per request.

    tile = (tf, tm): a 128-byte line holds tf x tm quads of a plane ((8, 1):
    the row-major layout; (4, 2), (2, 4): tiled alternatives).  march =
    "slabs" (the kernel's slabs of width D from the first sample) or "rows"
    (slabs aligned to the depth axis's unit rows, every lane taking its
    samples in the row one request at a time, so a request's lanes share a
    row)."""
    rng = np.random.default_rng(seed)
    nx, ny, _ = geo["n_voxel"]
    nu, nv = geo["n_det"]
    cw = 32 // ag
    requests = warp_lines = half_lines = lanes = 0
    for _ in range(n_warps):
        a = int(rng.integers(0, len(angles) - ag + 1))
        row = int(rng.integers(0, nv))
        p0 = int(rng.integers(0, nu // cw)) * cw
        group = angles[a:a + ag]
        if len({layout(t) for t in group}) > 1:
            continue
        parts = [rays(geo, t, np.arange(p0, p0 + cw, dtype=float), row) for t in group]
        x0 = np.concatenate([q[0] for q in parts])
        dx = np.concatenate([q[1] for q in parts])
        K = np.concatenate([q[2] for q in parts])
        lay = parts[0][3]
        pf = (ny if lay else nx) + 2 * PAD
        pm = (nx if lay else ny) + 2 * PAD
        slot = np.arange(len(K))  # angle-major: slot // cw is the angle
        lane = slot if order == "blocked" else (slot % cw) * ag + slot // cw
        act = K > 0
        if not act.any():
            continue
        if np.all(dx[act, 1] > 0):
            sgn = 1.0
        elif np.all(dx[act, 1] < 0):
            sgn = -1.0
        else:
            continue  # mixed directions: the kernel's per-lane loop, not the march
        y0, dy = sgn * x0[:, 1], sgn * dx[:, 1]
        D = dy[act].min()
        Y0 = y0[act].min()
        Y1 = (y0 + (K - 1) * dy)[act].max()
        k = np.zeros(len(K), int)
        tf, tm = tile

        def request(take):
            nonlocal requests, lanes, warp_lines, half_lines
            cell = np.floor(x0[take] + k[take][:, None] * dx[take]).astype(np.int64)
            if (tf, tm) == (8, 1):
                ln = ((cell[:, 2] * pm + cell[:, 1]) * pf + cell[:, 0]) * QUAD // LINE
            else:  # lines of tf x tm quads
                ptf, ptm = (pf + tf - 1) // tf, (pm + tm - 1) // tm
                ln = (cell[:, 2] * ptm + cell[:, 1] // tm) * ptf + cell[:, 0] // tf
            half = lane[take] // 16
            requests += 1
            lanes += int(take.sum())
            warp_lines += len(np.unique(ln))
            half_lines += sum(len(np.unique(ln[half == h])) for h in np.unique(half))
            k[take] += 1

        if march == "slabs":
            for j in range(1, int((Y1 - Y0) / D) + 2):
                take = act & (k < K) & (y0 + k * dy < Y0 + j * D)
                if take.any():
                    request(take)
        else:
            bound = np.floor(Y0)
            while bound <= Y1:
                bound += 1.0
                while True:
                    take = act & (k < K) & (y0 + k * dy < bound)
                    if not take.any():
                        break
                    request(take)
    return {"ag": ag, "order": order, "tile": list(tile), "march": march, "requests": requests,
            "lines_per_request": warp_lines / max(requests, 1),
            "halfwarp_lines_per_request": half_lines / max(requests, 1),
            "lanes_per_request": lanes / max(requests, 1)}


def main():
    from . import synth

    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", default="cgls_512")
    ap.add_argument("--warps", type=int, default=400)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--variants", action="store_true",
                    help="also tiled quad lines and row-aligned marching")
    a = ap.parse_args()
    geo, ang = synth.workload(a.workload)
    for ag, order in ((1, "blocked"), (2, "blocked"), (2, "interleaved")):
        print(json.dumps(replay(geo, ang, ag, order, a.warps, a.seed)))
    if a.variants:
        for tile in ((4, 2), (2, 4)):
            print(json.dumps(replay(geo, ang, 2, "interleaved", a.warps, a.seed, tile=tile)))
        print(json.dumps(replay(geo, ang, 2, "interleaved", a.warps, a.seed, march="rows")))


if __name__ == "__main__":
    main()
