"""The exchange steps between processes (one GPU each) of a multi-GPU SLMC run.

Chains are independent, so the cumulative updates (Eq. (6)) need no communication; the one
step that couples processes is the regression of the effective model (Eq. (5)), which fits
all processes' configurations together. Each process reduces its own configurations to a
fixed-size partial state in libslmc (`slmc_fit_eff_state`), the states are all-gathered
here (64 doubles per process, rank order), and every process merges the same stacked states
in libslmc (`slmc_fit_eff_merge`), so all processes obtain identical couplings. Measurement
accumulators (acceptance counts, S(pi, pi) sums) are summed across processes.
Works with any torch.distributed backend (NCCL on GPUs, gloo on CPU tensors)."""
import torch


def _world(group=None):
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return 1
    return dist.get_world_size(group)


def gather_states(state, group=None):
    """All-gather of one 1-D partial state per process -> [world, len(state)] in rank order."""
    state = state.reshape(-1).contiguous()
    world = _world(group)
    if world == 1:
        return state.reshape(1, -1)
    import torch.distributed as dist
    parts = [torch.empty_like(state) for _ in range(world)]
    dist.all_gather(parts, state, group=group)
    return torch.stack(parts)


def fit_eff_distributed(ctx, xs, lnw, group=None):
    """Eq. (5) over the configurations of all processes: (J [6], rms residual [1]), identical on
    every process. `ctx` is a libslmc Context (or anything with the same two methods)."""
    state = ctx.fit_eff_state(xs, lnw)
    return ctx.fit_eff_merge(gather_states(state, group))


def sum_over_processes(t, group=None):
    """In-place sum of an accumulator tensor over all processes; returns it."""
    if _world(group) > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t
