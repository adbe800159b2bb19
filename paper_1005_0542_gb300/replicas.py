"""Multi-GPU by replicas: every rank solves its own shot; no data-path collective.

The method's sources and shots are independent, so N GPUs run N replica shots (weak scaling).
The only communication is the benchmark's barrier and the max-over-ranks of the timed region.
"""


def replica_source(base_source, rank, nx, spacing=64):
    """Source of replica `rank`: the base source shifted along its row by rank * spacing nodes."""
    ix, iz = base_source
    return ((ix + spacing * rank) % nx, iz)


def whole_job_rate(local_seconds, units_per_rank, world, dist=None, device=None):
    """Aggregate throughput: units of all ranks over the slowest rank's time."""
    t = float(local_seconds)
    if dist is not None and world > 1:
        import torch
        x = torch.tensor([t], dtype=torch.float64, device=device or "cpu")
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return world * units_per_rank / t, t
