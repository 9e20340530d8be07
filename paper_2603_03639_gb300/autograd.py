"""torch.autograd form of the robust-control objective.

``fidelity(u, ctx)`` returns the ensemble-averaged fidelity F(u) (Sec. II) as
a differentiable scalar of the control tensor u[K][C][N] (CUDA, float64).
Its backward is the hand-written costate (adjoint) kernel of App. A: the
trajectory kernel propagates the target backwards through the truncated
layers.  The forward layer states it needs are read from a packed history
written during the forward pass at their actual bond dimensions (the default:
nothing is recomputed).  Each CTA's work region is sized for about
2 sqrt(L) full-capacity MPS (L truncated layers); a trajectory whose packed
history outgrows it is redone on the fallback path, which keeps checkpoints
every ``checkpoint_every`` slices (about sqrt(L) layers by default) and
recomputes each segment, so device memory stays bounded by the sqrt-sized
region either way (results are bitwise the same on both paths).

When the graph requires a gradient, the adjoint runs in the same device
launch as the forward pass (one forward and one costate sweep per
trajectory, instead of a second forward in a separate backward launch) and
its result dF/du is held until ``backward``; otherwise only the forward pass
runs.  Everything is stream-ordered on the context's stream;
no host synchronisation happens in either direction.
"""
import torch

from .tnrc import Context


class TNRCFidelity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u: torch.Tensor, tn: Context):
        if not (u.is_cuda and u.dtype == torch.float64 and u.is_contiguous()):
            raise TypeError("controls must be a contiguous CUDA float64 tensor")
        if tuple(u.shape) != (tn.K, tn.C, tn.N):
            raise ValueError("controls must have shape (K, C, N) = %r" % ((tn.K, tn.C, tn.N),))
        if tn.stream != torch.cuda.current_stream(u.device).cuda_stream:
            raise RuntimeError("the tnrc context must be ordered on torch's current stream")
        F = torch.empty(1, dtype=torch.float64, device=u.device)
        tn.set_controls_dev(u.data_ptr())
        if ctx.needs_input_grad[0]:
            g = torch.empty_like(u)
            tn.evaluate_dev(F.data_ptr(), g.data_ptr())
            ctx.save_for_backward(g)
        else:
            tn.evaluate_dev(F.data_ptr())
        return F[0]

    @staticmethod
    def backward(ctx, gF):
        (g,) = ctx.saved_tensors
        return gF * g, None


def fidelity(u: torch.Tensor, tn: Context) -> torch.Tensor:
    """Differentiable ensemble fidelity of controls ``u`` on context ``tn``
    (noise must have been set or sampled on ``tn``)."""
    return TNRCFidelity.apply(u, tn)
