"""Test-harness helper: the oracle's snapshot-misfit gradient with recomputation.

The FP64 oracle's adjoint is autograd through its plain step function; over a few
hundred steps on a 256^2 lattice the tape would not fit in host memory.  This runs the
same oracle functions in segments under torch.utils.checkpoint (the segment's steps are
recomputed during the backward pass), which changes only what autograd stores, not the
arithmetic.  Test infrastructure: only the tests import it.
"""
import torch
from torch.utils.checkpoint import checkpoint

from oracle import lbm_oracle as O


def loss_and_grad(pb, C0, snap_steps, obs, seg=50):
    """(loss, dL/d[alpha, p, D_diag, u]) of sum_k |C(t_k) - obs_k|^2, as
    oracle.lbm_oracle.loss_and_grad, with every `seg` steps checkpointed."""
    d = pb.d
    DT = torch.float64
    alpha = torch.tensor(pb.alpha, dtype=DT, requires_grad=True)
    p = torch.tensor(pb.p, dtype=DT, requires_grad=True)
    Dd = torch.tensor([pb.D[i][i] for i in range(d)], dtype=DT, requires_grad=True)
    u = torch.tensor(pb.u, dtype=DT, requires_grad=True)
    ops = O.Operators(pb, alpha=alpha, p=p, D=torch.diag(Dd), u=u)
    obs_t = torch.as_tensor(obs, dtype=DT)

    def advance(f, n):
        for _ in range(n):
            f = O.step(ops, f)
        return f

    f = O.init_populations(ops, torch.as_tensor(C0, dtype=DT))
    loss = torch.zeros((), dtype=DT)
    t = 0
    for k, ts in enumerate(snap_steps):
        while t < ts:
            n = min(seg, ts - t)
            f = checkpoint(advance, f, n, use_reentrant=False)
            t += n
        r = O.concentration(f) - obs_t[k]
        loss = loss + (r * r).sum()
    loss.backward()
    return float(loss.detach()), torch.cat([alpha.grad, p.grad, Dd.grad, u.grad])
