"""torch.autograd.Function around the library's PPO loss and its hand-written backward.

The loss is the clipped PPO objective of Sec. 2.2 / Table 3 on one minibatch: clipped surrogate,
clipped value loss (coefficient 1) and entropy bonus (coefficient 0.01).  forward sets the
learner's parameters (rl_set_params) and runs rl_ppo_loss_grad, which returns the loss and, from
the same kernels, the gradient derived by hand (heads, ELU layers, linear layers).  The loss comes
back as a 0-d tensor; the gradient is kept for backward.  backward hands that gradient to autograd,
multiplied by the incoming gradient of the loss (the chain-rule product autograd requires; 1 when
the loss is the root of the graph).  The loss and its gradient are computed entirely by the
library's kernels.
"""
import torch

from . import api


class PPOLoss(torch.autograd.Function):
    """loss = PPOLoss.apply(params, learner, batch).

    params: CUDA fp32 [rl_param_count] in the flat layout of rl_get_params.  learner: an
    api.Learner (its parameters are overwritten).  batch: dict of CUDA tensors with the keys obs,
    actions, logp_old, mu_old, log_std_old, v_old, adv, ret (layouts of rl_ppo_loss_grad; M rows,
    M a multiple of 64 and at most the learner's minibatch size)."""

    @staticmethod
    def forward(ctx, params, learner, batch):
        if params.dtype != torch.float32 or not params.is_cuda or params.numel() != learner.n_params:
            raise api.RLError("PPOLoss: params must be a CUDA float32 vector of rl_param_count values")
        learner.set_params(params.detach())
        grad = torch.empty(learner.n_params, dtype=torch.float32, device=params.device)
        stats = torch.empty(api.RL_NSTATS, dtype=torch.float32, device=params.device)
        api.rl_ppo_loss_grad(learner.ctx, batch["obs"], batch["actions"], batch["logp_old"], batch["mu_old"],
                             batch["log_std_old"], batch["v_old"], batch["adv"], batch["ret"], grad, stats)
        ctx.save_for_backward(grad)
        return stats[0].clone()

    @staticmethod
    def backward(ctx, grad_loss):
        (grad,) = ctx.saved_tensors
        return grad_loss * grad, None, None


def ppo_loss(params, learner, batch):
    """The minibatch PPO loss as a differentiable function of the flat parameters."""
    return PPOLoss.apply(params, learner, batch)
