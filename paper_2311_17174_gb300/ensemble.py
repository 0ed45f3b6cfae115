"""One ensemble spread over several GPUs (one process per GPU).

The paper samples its posterior with the parallel stretch move (Sec. 3,
"Posterior sampling": emcee, after Goodman & Weare 2010): the two halves of
the ensemble are updated in turn, and the walkers of a half are independent
given the other half.  So each rank owns a contiguous block of each half --
block r of a half of n_s walkers starting at s0 is
[s0 + floor(r n_s / R), s0 + floor((r + 1) n_s / R)) -- keeps a replica of
the whole ensemble (and of the dataset) on its GPU, and for each half:

  1. moves its own block (``emri_stretch_half``, on its GPU);
  2. all-gathers every rank's block (positions, log-posterior, acceptance),
     so every replica holds the updated half before the other half moves.

That all-gather is the data path's only exchange: 8 (P + 2) bytes per walker
per half-step.  The result is bit for bit the ensemble step of one GPU.

The host logic here is independent of where a block is moved and how blocks
are exchanged: ``sharded_stretch_step`` takes both as callables, so the same
code runs with the library on GPUs and NCCL, or with any other block update
and collective.
"""
from __future__ import annotations


def shard_block(w: int, world: int, rank: int, half: int) -> tuple[int, int]:
    """Walkers [k0, k1) of ``half`` (0: [0, W/2), 1: [W/2, W)) owned by ``rank``."""
    h = w // 2
    s0, n = (0, h) if half == 0 else (h, w - h)
    return s0 + (n * rank) // world, s0 + (n * (rank + 1)) // world


def sharded_stretch_step(theta, lnp, accepted, rank: int, world: int, move_block, all_gather):
    """One ensemble step with the walkers sharded over ``world`` ranks.

    theta [P][W], lnp [W], accepted [W]: torch tensors holding the whole
    ensemble (a replica per rank; updated in place).  ``move_block(half, k0,
    k1)`` moves walkers k0..k1-1 of the half in place.  ``all_gather(block,
    widths)`` exchanges this rank's block, a float64 tensor [P + 2][k1 - k0]
    (positions, lnp, accepted), and returns every rank's block in rank order
    (widths: the block widths of all ranks).
    """
    import torch

    w = theta.shape[1]
    for half in (0, 1):
        k0, k1 = shard_block(w, world, rank, half)
        move_block(half, k0, k1)
        block = torch.cat([theta[:, k0:k1], lnp[None, k0:k1], accepted[None, k0:k1].to(theta.dtype)], 0)
        widths = [shard_block(w, world, r, half)[1] - shard_block(w, world, r, half)[0] for r in range(world)]
        for r, part in enumerate(all_gather(block, widths)):
            r0, r1 = shard_block(w, world, r, half)
            theta[:, r0:r1] = part[:-2]
            lnp[r0:r1] = part[-2]
            accepted[r0:r1] = part[-1].to(accepted.dtype)


def dist_all_gather(block, widths):
    """torch.distributed all-gather of blocks of unequal width (each padded
    to the widest); on the current stream for NCCL."""
    import torch
    import torch.distributed as dist

    if len(widths) == 1:
        return [block]
    wmax = max(widths)
    buf = torch.zeros((block.shape[0], wmax), dtype=block.dtype, device=block.device)
    buf[:, :block.shape[1]] = block
    outs = [torch.empty_like(buf) for _ in widths]
    dist.all_gather(outs, buf)
    return [o[:, :m] for o, m in zip(outs, widths)]


class ShardedEnsemble:
    """The ensemble step of ``emri_stretch_step`` with this rank's blocks
    moved on its GPU through ``emri_stretch_half`` and the blocks exchanged
    with ``torch.distributed`` (NCCL between GPUs)."""

    def __init__(self, ctx, ds, opts, cfg, rank: int, world: int, all_gather=dist_all_gather):
        self.ctx, self.ds, self.opts, self.cfg = ctx, ds, opts, cfg
        self.rank, self.world, self.all_gather = rank, world, all_gather

    def step(self, theta, lnp, u, accepted):
        """theta [16][W], lnp [W], u [3][W] (uniforms), accepted [W] int32:
        device tensors of the whole ensemble, replicated on every rank."""
        def move(half, k0, k1):
            self.ctx.stretch_half(self.ds, theta, lnp, self.opts, self.cfg, u, half, k0, k1, accepted)

        sharded_stretch_step(theta, lnp, accepted, self.rank, self.world, move, self.all_gather)
