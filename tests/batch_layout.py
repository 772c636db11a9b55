"""Workspace layout of fbp_batched / fbp_batched_scans, restated for the
host tests: the per-item padded table of the staged batch units.

An item runs staged units when its rows' geometry has the 90-degree orbit
symmetry with T x T tiles (T = 32 for FP32 rows, 64 for 16-bit rows: K
even, K * angle_step = pi, a centred detector, n a multiple of 2T) and its
window W = 2H + 1, H = ceil(alpha * sqrt(2) * (T - 1) / 2) + 2, padded to a
multiple of 8 entries, is at most 72 (FP32) / 104 (16-bit).  Its table
holds K/2 rows of Ep 16-byte entries (two planes for FP32 rows): P_lo zero
entries before segment -1, enough after segment D-1 for the window of every
orbit tile, whose centre lies within alpha (n - T) / sqrt 2 of the detector
centre."""
import math


def align256(n):
    return (n + 255) // 256 * 256


def staged_item_geom(K, D, N, alpha=1.0, det_center=None, angle_step=None, f32=True):
    """(H, W, Wp, P_lo, Ep) of the item's padded table, or None if the item
    does not run staged units."""
    T = 32 if f32 else 64
    c = 0.5 * (D - 1) if det_center is None else det_center
    step = math.pi / K if angle_step is None else angle_step
    if K % 2 or N % (2 * T) or abs(step * K - math.pi) > 1e-9 * math.pi or abs(c - 0.5 * (D - 1)) > 1e-9 * (1 + D):
        return None
    h = 0.5 * (T - 1)
    H = math.ceil(alpha * math.sqrt(h * h * 2)) + 2
    W = 2 * H + 1
    Wp = (W + 7) // 8 * 8
    if Wp > (72 if f32 else 104):
        return None
    R = alpha * (N - T) / math.sqrt(2.0) * (1 + 1e-12) + 1e-6
    lo, hi = math.floor(c - R), math.floor(c + R)
    P_lo = max(0, H + 1 - lo)
    Ep = max(D + 1, hi + H + 4) + P_lo
    return H, W, Wp, P_lo, Ep


def staged_table_bytes(K, D, N, alpha=1.0, det_center=None, angle_step=None, f32=True):
    """Bytes of the item's padded table, or 0 if it does not run staged units."""
    geom = staged_item_geom(K, D, N, alpha, det_center, angle_step, f32)
    if geom is None:
        return 0
    Ep = geom[4]
    return align256((K // 2) * Ep * 16 * (2 if f32 else 1))
