"""Data-parallel training of the learned correction's network (one process per GPU).

Each rank draws its own minibatches from its own shard of the training rows, computes the
gradient of its batch's mean loss on its GPU (hl_mlp_loss_grad), and the ranks average the
gradients in place (an all-reduce on the network's stream) before every Adam step, so that
replicas that start from the same weights stay identical: with equal batch sizes the
average is the gradient of the mean loss over all ranks' rows.  The learned correction
itself (features, targets, the FP64 correction inside hl_step) runs through the C ABI."""
from __future__ import annotations


def shard_range(n: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous share [lo, hi) of n items for rank (the first n % world ranks get one more)."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard arguments")
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def allreduce_mean_(t, dist=None) -> None:
    """t <- mean of t over the ranks of the default process group (in place).  NCCL reduces
    on the current CUDA stream, so callers keep the network on that stream."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return
    dist.all_reduce(t)
    t.div_(dist.get_world_size())


def train(net, X_pool, T_pool, iters: int, batch: int, lr, seed: int, dist=None) -> None:
    """iters data-parallel Adam steps of batch rows per rank.  X_pool/T_pool: this rank's
    training rows on its GPU; lr(it) the learning rate of step it; the network must be on
    torch's current stream (hl_mlp_set_stream) and identical on every rank at the start."""
    import torch

    from . import hl

    rank = dist.get_rank() if dist is not None and dist.is_initialized() else 0
    grads = hl.hl_mlp_grad_tensor(net)
    Xb = torch.empty((batch, hl.HL_MLP_IN), dtype=torch.float32, device=X_pool.device)
    Tb = torch.empty((batch, hl.HL_MLP_OUT), dtype=torch.float32, device=X_pool.device)
    for it in range(iters):
        hl.hl_mlp_sample(net, X_pool, T_pool, batch, seed + 7919 * rank, it, Xb, Tb)
        hl.hl_mlp_loss_grad(net, Xb, Tb, batch, want_loss=False)
        allreduce_mean_(grads, dist)
        hl.hl_mlp_adam_step(net, lr(it))
