"""torch.autograd.Function over the library's quality functional.

forward(xy, m, tri) = sum over elements of the Vasilevskii-Lipnikov quality
(Sec. 2.2) in the element-mean metric; backward runs the library's
hand-written reverse-mode kernel for d/d(xy) and d/d(m) and scales it by the
incoming gradient.  xy: (nv, 2) float64 CUDA, m: (nv, 3) float64 CUDA,
tri: (ne, 3) int32 CUDA (counter-clockwise).
"""
import torch

from . import pm


class QualityFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xy, m, tri):
        xy = xy.contiguous()
        m = m.contiguous()
        tri = tri.contiguous()
        q = torch.empty(1, dtype=torch.float64, device=xy.device)
        stream = torch.cuda.current_stream(xy.device).cuda_stream
        pm.quality_arrays_dev(xy, m, tri, q, None, None, stream=stream)
        ctx.save_for_backward(xy, m, tri)
        return q[0]

    @staticmethod
    def backward(ctx, grad):
        xy, m, tri = ctx.saved_tensors
        q = torch.empty(1, dtype=torch.float64, device=xy.device)
        dxy = torch.empty_like(xy)
        dm = torch.empty_like(m)
        stream = torch.cuda.current_stream(xy.device).cuda_stream
        pm.quality_arrays_dev(xy, m, tri, q, dxy, dm, stream=stream)
        return grad * dxy, grad * dm, None


def quality(xy, m, tri):
    return QualityFunction.apply(xy, m, tri)
