"""torch.autograd wrappers of the differentiable extension (C ABI calls only).

``lse_statistic(x, plan, tau)`` returns Y[segment, width], the logsumexp
relaxation (temperature tau) of the per-(segment, width) maximum boxcar
power of the series in ``x`` (the plan's layout); its backward is the
library's hand-written adjoint (pulscan_lse_backward).  ``inject(noise,
template, amp, plan)`` builds x = noise + amp * template per series with a
backward to ``amp`` (pulscan_amplitude_grad).  Tensors only provide device
memory and the stream; every step runs in the library's kernels.
"""
import torch

from . import _check, _stream, load


class _LogSumExp(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, plan, tau):
        lib = load()
        dev = x.device
        x = x.contiguous()
        spec = torch.empty(plan.spec_floats, dtype=torch.float32, device=dev)
        power = torch.empty(plan.power_floats, dtype=torch.float32, device=dev)
        stats = torch.empty(4 * plan.total_segments, dtype=torch.float32, device=dev)
        sel = torch.empty(8 * plan.total_segments, dtype=torch.float32, device=dev)
        y = torch.empty(plan.total_segments * plan.z_max, dtype=torch.float32, device=dev)
        ylo = torch.empty_like(y)
        _check(lib.pulscan_lse_forward(plan._h, x.data_ptr(), spec.data_ptr(), power.data_ptr(), stats.data_ptr(),
                                       sel.data_ptr(), y.data_ptr(), ylo.data_ptr(), float(tau), _stream(None)))
        ctx.save_for_backward(spec, power, stats, sel, y, ylo)
        ctx.plan = plan
        ctx.tau = float(tau)
        return y.view(plan.total_segments, plan.z_max)

    @staticmethod
    def backward(ctx, gy):
        lib = load()
        spec, power, stats, sel, y, ylo = ctx.saved_tensors
        plan = ctx.plan
        gy = gy.contiguous().view(-1)
        gx = torch.empty(plan.x_floats, dtype=torch.float32, device=gy.device)
        _check(lib.pulscan_lse_backward(plan._h, spec.data_ptr(), power.data_ptr(), stats.data_ptr(),
                                        sel.data_ptr(), y.data_ptr(), ylo.data_ptr(), gy.data_ptr(), gx.data_ptr(),
                                        ctx.tau, _stream(None)))
        return gx, None, None


class _Inject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, noise, template, amp, plan):
        lib = load()
        noise, template, amp = noise.contiguous(), template.contiguous(), amp.contiguous()
        x = torch.empty_like(noise)
        _check(lib.pulscan_inject(plan._h, noise.data_ptr(), template.data_ptr(), amp.data_ptr(), x.data_ptr(),
                                  _stream(None)))
        ctx.save_for_backward(template)
        ctx.plan = plan
        ctx.n_amp = amp.numel()
        return x

    @staticmethod
    def backward(ctx, gx):
        lib = load()
        (template,) = ctx.saved_tensors
        gx = gx.contiguous()
        gamp = torch.empty(ctx.n_amp, dtype=torch.float32, device=gx.device)
        _check(lib.pulscan_amplitude_grad(ctx.plan._h, gx.data_ptr(), template.data_ptr(), gamp.data_ptr(),
                                          _stream(None)))
        return None, None, gamp, None


def lse_statistic(x, plan, tau=0.1):
    """Y[segment, width] (differentiable in x)."""
    return _LogSumExp.apply(x, plan, tau)


def inject(noise, template, amp, plan):
    """x = noise + amp[series] * template (differentiable in amp)."""
    return _Inject.apply(noise, template, amp, plan)
