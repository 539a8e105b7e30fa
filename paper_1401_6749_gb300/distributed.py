"""Source-parallel TSM over several GPUs (one process per GPU).

The work of the method shards over independent stochastic sources (Sec. 2):
rank g runs its own N_HP + N_LP sources with source indices starting at
g (N_HP + N_LP), so no two ranks draw the same Z4 vector and no data moves
while the sources are solved and contracted.  The only exchange is the final
gather of the per-source loop values (kilobytes per source) that the global
TSM combination (Eq. 4) needs: the HP sets, the LP values of the HP sources
and the LP-only sets of all ranks, concatenated in rank order (= source order).
"""
import torch


def rank_sources(rank, n_hp, n_lp):
    """First source index of a rank and its number of sources (weak scaling)."""
    n = int(n_hp) + int(n_lp)
    return int(rank) * n, n


def gather_tsm_sets(dist, hp, lp, n_hp, group=None):
    """All-gather the per-source loops of every rank.

    hp: [n_hp, len] HP loops of this rank's HP sources; lp: [n_hp + n_lp, len]
    LP loops of all its sources (the first n_hp are the HP sources).  Returns
    (hp_all, lp_on_hp_all, lp_only_all) over all ranks in rank order (every rank
    receives them).  Works with the gloo (CPU tensors) and NCCL (CUDA tensors)
    backends.
    """
    world = dist.get_world_size(group)
    hp_list = [torch.empty_like(hp) for _ in range(world)]
    lp_list = [torch.empty_like(lp) for _ in range(world)]
    dist.all_gather(hp_list, hp.contiguous(), group=group)
    dist.all_gather(lp_list, lp.contiguous(), group=group)
    hp_all = torch.cat(hp_list[:], dim=0)
    lp_on_hp = torch.cat([x[:n_hp] for x in lp_list], dim=0)
    lp_only = torch.cat([x[n_hp:] for x in lp_list], dim=0)
    return hp_all, lp_on_hp, lp_only
