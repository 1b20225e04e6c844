"""Host-side work partitioning across ranks (one process per GPU).

The momenta are independent (Sec. III: "each momentum is independent"), so the
path shards without any data exchange: whole solves (independent pulse
samples or requests) go to ranks round-robin, or one large grid is cut into
bands of rows.  The only cross-rank steps are host-side: the max of the
per-rank wall times, and the fixed-order (rank-order) sum of per-band density
contributions.
"""
from __future__ import annotations


def sample_for(step: int, rank: int, world: int, n_samples: int, offset: int = 0) -> int:
    """Round-robin: the sample rank ``rank`` solves at benchmark step ``step``."""
    return (offset + step * world + rank) % n_samples


def row_band(ny: int, rank: int, world: int) -> tuple[int, int]:
    """Rows [r0, r1) of an ny-row grid owned by ``rank`` (sizes differ by <= 1)."""
    base, extra = divmod(ny, world)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def band_grid(grid: dict, rank: int, world: int) -> dict:
    """The sub-grid of a rank's row band, with its own p_y range (cell-centred
    nodes of the band coincide with the full grid's rows up to rounding)."""
    r0, r1 = row_band(grid["ny"], rank, world)
    lo, hi = grid["py"]
    h = (hi - lo) / grid["ny"]
    return {"nx": grid["nx"], "ny": r1 - r0, "px": grid["px"], "py": (lo + r0 * h, lo + r1 * h)}


def combine_densities(parts: list[float]) -> float:
    """Sum of per-band densities in rank order (deterministic)."""
    total = 0.0
    for p in parts:
        total += p
    return total
