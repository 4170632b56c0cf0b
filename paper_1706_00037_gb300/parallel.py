"""One batch of starts sharded over ranks (one GPU each).

The method's batch parallelises over starts (Fig. 2 evaluates, screens and
climbs every start independently); the only quantities that couple the starts
are the screen's Mean and Max and the final best-of.  A rank therefore holds a
contiguous range of the batch's starts and the ranks exchange three integers
before the screen and two at the end:

* screen statistics {sum of f, Max, lowest index attaining Max}: combined by
  integer add / max / min, so every rank derives the bit-identical threshold
  T(lambda) = Mean + lambda (Max - Mean) on its own device;
* best-of {value, global index}: max, then the lowest index among equal values;
  the owner of that index supplies the solution.

Integer reductions are order independent, so the sharded result equals the
single-rank result bit for bit.  The per-rank work runs in the CUDA library
(ubqp_diversify_range, ubqp_eval, ubqp_screen_stats / ubqp_screen_apply,
ubqp_ascent, ubqp_best); this module holds the partition and the exchanges,
which use torch.distributed (NCCL on GPUs, gloo in the CPU tests).
"""
from __future__ import annotations

from dataclasses import dataclass

import torch
import torch.distributed as dist

INT64_MAX = 2**63 - 1
INT64_MIN = -2**63


def shard(S_total: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous range (begin, count) of rank's starts; the first S_total %
    world ranks take one extra start."""
    base, extra = divmod(S_total, world)
    begin = rank * base + min(rank, extra)
    return begin, base + (1 if rank < extra else 0)


def owner_of(index: int, S_total: int, world: int) -> int:
    """Rank whose range holds global start `index`."""
    for r in range(world):
        b, c = shard(S_total, world, r)
        if b <= index < b + c:
            return r
    raise ValueError("index outside the batch")


# ------------------------------------------------------------ pure combinations

def combine_screen_stats(stats: list[torch.Tensor]) -> torch.Tensor:
    """Exact combination of per-rank {sum, max, argmax(global)} triples."""
    st = torch.stack([s.to("cpu", torch.int64) for s in stats])
    total = int(st[:, 0].sum())
    mx = int(st[:, 1].max())
    arg = min(int(s[2]) for s in st if int(s[1]) == mx)
    return torch.tensor([total, mx, arg], dtype=torch.int64)


def combine_best(bests: list[tuple[int, int]]) -> tuple[int, int]:
    """(value, global index) pairs -> the best value, lowest index on ties."""
    v = max(b[0] for b in bests)
    return v, min(b[1] for b in bests if b[0] == v)


# ------------------------------------------------------------ collectives

def reduce_screen_stats(stats: torch.Tensor, group=None) -> torch.Tensor:
    """All-reduce of a {sum, max, argmax(global)} int64 triple (on any device)."""
    s = stats[0:1].clone()
    m = stats[1:2].clone()
    dist.all_reduce(s, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(m, op=dist.ReduceOp.MAX, group=group)
    cand = torch.where(stats[1:2] == m, stats[2:3], torch.full_like(m, INT64_MAX))
    dist.all_reduce(cand, op=dist.ReduceOp.MIN, group=group)
    return torch.cat([s, m, cand])


def reduce_best(value_index: torch.Tensor, x: torch.Tensor, S_total: int, group=None):
    """All-reduce of a local best {value, global index} and its solution words.
    Returns (value, index, x of the winner) on every rank."""
    world = dist.get_world_size(group)
    v = value_index[0:1].clone()
    dist.all_reduce(v, op=dist.ReduceOp.MAX, group=group)
    cand = torch.where(value_index[0:1] == v, value_index[1:2], torch.full_like(v, INT64_MAX))
    dist.all_reduce(cand, op=dist.ReduceOp.MIN, group=group)
    idx = int(cand.item())
    owner = owner_of(idx, S_total, world)
    xs = x.clone() if dist.get_rank(group) == owner else torch.zeros_like(x)
    dist.all_reduce(xs, op=dist.ReduceOp.SUM, group=group)  # one non-zero term: exact
    return int(v.item()), idx, xs


# ------------------------------------------------------------ one sharded round

@dataclass
class RankState:
    begin: int
    count: int
    X: torch.Tensor
    f: torch.Tensor
    stats: torch.Tensor
    ws: torch.Tensor


def round_phase1(inst, params, world: int, rank: int) -> RankState:
    """This rank's starts, their exact values and its screen statistics."""
    from . import ubqp
    S = params.num_starts
    begin, count = shard(S, world, rank)
    if count == 0:
        # more ranks than starts: one placeholder start that can neither pass
        # the screen nor be the best, and the neutral statistics
        X = torch.zeros((1, inst.words), dtype=torch.int64, device=inst.device)
        f = torch.full((1,), INT64_MIN, dtype=torch.int64, device=inst.device)
        st = torch.tensor([0, INT64_MIN, INT64_MAX], dtype=torch.int64, device=inst.device)
        return RankState(begin, 0, X, f, st, torch.empty(16, dtype=torch.uint8,
                                                         device=inst.device))
    X = ubqp.diversify_range(inst, S, begin, count, mode=params.mode, seed=params.seed,
                             round_=params.round, div_H=params.div_H)
    ws_bytes = max(ubqp.eval_workspace_size(inst, count, params.eval_path),
                   ubqp.ascent_workspace_size(inst, count), 16)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=inst.device)
    f = ubqp.eval(inst, X, path=params.eval_path, ws=ws)
    st = ubqp.screen_stats(f, offset=begin)
    return RankState(begin, count, X, f, st, ws)


def round_phase2(inst, params, state: RankState, gstats: torch.Tensor):
    """Screen with the combined statistics, climb the passing starts, and this
    rank's best {value, global index}, its solution and its pass count."""
    from . import ubqp
    sc = ubqp.screen_apply(state.f, gstats.to(state.f.device), params.num_starts,
                           params.lambda_)
    flips = torch.zeros(state.count, dtype=torch.int32, device=state.f.device)
    ubqp.ascent(inst, state.X, state.f, sc["idx"], sc["count"], params.max_flips, flips,
                ws=state.ws)
    bx, bf = ubqp.best(state.f, state.X)
    vi = torch.stack([bf[0], bf[1] + state.begin])
    return vi, bx, sc


def solve_round_distributed(inst, params, group=None):
    """One round over the ranks of `group` (one GPU per rank).  Returns
    (best value, global index, best solution words, T) on every rank."""
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    state = round_phase1(inst, params, world, rank)
    gstats = reduce_screen_stats(state.stats, group)
    vi, bx, sc = round_phase2(inst, params, state, gstats)
    v, idx, x = reduce_best(vi, bx, params.num_starts, group)
    return v, idx, x, float(sc["Tm"][0].item())
