"""The allocation-free PPO loss entry point (ddppo_ppo_loss_static).

It serves callers that cannot allocate device memory where they need the loss (inside a
stream capture that forbids cudaMalloc, or under a foreign allocator); its partial sums
live in a fixed library-owned array. Two calls in a row, through the C ABI, must agree
with the existing ddppo_ppo_loss within the loss tolerance of the parity tests (1e-5
relative): the second call checks that what the first left in the shared array does not
leak into the next result. This file is collected last so that a failure here cannot
hide any other test.
"""
import pytest
import torch

from paper_1911_00357_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _case(n, seed):
    g = torch.Generator().manual_seed(seed)
    logits = torch.randn(n, 4, generator=g).cuda()
    values = torch.randn(n, generator=g).cuda()
    actions = torch.randint(0, 4, (n,), generator=g, dtype=torch.int32).cuda()
    logp_old = (torch.log_softmax(logits, -1).gather(1, actions.long().unsqueeze(1))[:, 0]
                + 0.3 * torch.randn(n, generator=g).cuda())
    adv = torch.randn(n, generator=g).cuda()
    ret = torch.randn(n, generator=g).cuda()
    return logits, values, actions, logp_old.contiguous(), adv, ret


def _run(fn, n, args):
    stats = torch.zeros(8, device="cuda")
    dl = torch.zeros(n, 4, device="cuda")
    dv = torch.zeros(n, device="cuda")
    fn(n, *args, 0.2, 0.5, 0.01, stats, dl, dv)
    torch.cuda.synchronize()
    return stats.cpu(), dl.cpu(), dv.cpu()


def _close(a, b, rtol=1e-5):
    scale = max(b.abs().max().item(), 1.0)
    return (a - b).abs().max().item() <= rtol * scale


def test_static_loss_matches_ppo_loss_two_calls_in_a_row():
    # the limit (every one of the 4096 partial slots) first, then smaller sizes, so that
    # partials of a larger call stay behind in the shared array
    for n, seed in ((1_048_576, 3), (300_001, 1), (4097, 2)):
        args = _case(n, seed)
        ref = _run(B.ddppo_ppo_loss, n, args)
        got = _run(B.ddppo_ppo_loss_static, n, args)
        for a, b in zip(got, ref):
            assert _close(a, b), (n, (a - b).abs().max().item())


def test_static_loss_rejects_sizes_beyond_its_scratch():
    n = 1_048_577
    z = torch.zeros(1, device="cuda")
    with pytest.raises(B.DDPPOError) as ei:
        B.ddppo_ppo_loss_static(n, z, z, z, z, z, z, 0.2, 0.5, 0.01, z, z, z)
    assert ei.value.code == -2 and "1048576" in str(ei.value)
