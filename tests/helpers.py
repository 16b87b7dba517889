"""Shared helpers of the GPU parity tests (no oracle arithmetic here)."""
import numpy as np

STATUS_MASK = 0x7F
TIE = 0x80


def split_lines(lines, grid):
    """CSR lines (torch) -> list of (n_i, 3) float64 arrays in index space."""
    off = lines.offsets.cpu().numpy()
    vert = lines.vertices.cpu().numpy().astype(np.float64)
    org = np.asarray(grid.origin, dtype=np.float64)
    sp = np.asarray(grid.spacing, dtype=np.float64)
    idx = (vert - org) / sp
    return [idx[off[i]:off[i + 1]] for i in range(len(off) - 1)]


def compare_lines(gpu_lines, grid, ref, tol, tie_cells=None, tie_eps_rel=1e-3, max_bad=0):
    """Compares GPU lines against oracle Lines.

    A line must have the same status and length as the oracle's, with every
    vertex within `tol` cells; a line whose lengths or statuses differ is
    accepted only as a boundary tie: the side that stopped first stopped by
    EXIT with its offending point less than `tie_cells` outside the domain, or
    by STAGNANT within `tie_eps_rel` of eps, and the common prefix matches.
    Returns a dict of statistics.
    """
    tie_cells = tol if tie_cells is None else tie_cells
    glines = split_lines(gpu_lines, grid)
    gst = gpu_lines.status.cpu().numpy() & STATUS_MASK
    gmg = gpu_lines.margin.cpu().numpy().astype(np.float64)
    n = len(glines)
    assert n == len(ref.length), (n, len(ref.length))
    max_err = 0.0
    errs = []
    ties = 0
    bad = []
    for i in range(n):
        g = glines[i]
        r = ref.line(i)
        same = (gst[i] == ref.status[i]) and (len(g) == len(r))
        k = min(len(g), len(r))
        e = float(np.abs(g[:k] - r[:k]).max()) if k else 0.0
        if not same:
            # the shorter side must have stopped at a tie
            def tie(st, mg):
                return (st == 2 and mg < tie_cells) or (st == 3 and mg < tie_eps_rel)
            if len(g) < len(r):
                ok = tie(gst[i], gmg[i])
            elif len(g) > len(r):
                ok = tie(ref.status[i], ref.margin[i])
            else:
                ok = tie(gst[i], gmg[i]) or tie(ref.status[i], ref.margin[i])
            if not ok:
                bad.append((i, int(gst[i]), len(g), int(ref.status[i]), len(r), float(gmg[i]), float(ref.margin[i])))
                continue
            ties += 1
        if e > tol:
            bad.append((i, "err", e))
            continue
        max_err = max(max_err, e)
        if k:
            errs.append(np.abs(g[:k] - r[:k]).max(axis=1))
    allerr = np.concatenate(errs) if errs else np.zeros(1)
    stats = dict(n=n, ties=ties, bad=bad, max_err=max_err, p99=float(np.percentile(allerr, 99)),
                 vertices=int(sum(len(x) for x in glines)))
    assert len(bad) <= max_bad, f"{len(bad)} mismatching lines (first: {bad[:5]}), stats {stats}"
    return stats
