"""Host-side work partitioning across ranks (one process per GPU).

The momenta are independent (Sec. III: every momentum carries its own spinor), so the
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
    """The band descriptor of a rank: the full grid (nx, ny, box) plus its rows
    [r0, r1).  Nodes are never re-derived from the band: the library
    (``dsp_create_band``, ``binding.Grid(..., rows=...)``) and the oracle both
    compute the full grid's nodes of those global rows, so a band's points are
    bitwise the full grid's."""
    r0, r1 = row_band(grid["ny"], rank, world)
    return {"nx": grid["nx"], "ny": grid["ny"], "px": grid["px"], "py": grid["py"],
            "rows": (r0, r1)}


def combine_densities(parts: list[float]) -> float:
    """Sum of per-band densities in rank order (deterministic)."""
    total = 0.0
    for p in parts:
        total += p
    return total
