"""encrypt_share_noalloc (the allocation-free variant of encrypt_share, for
callers that may not allocate device memory while they encrypt) gives the same
ciphertexts as encrypt_share, through the C ABI, on two calls in a row; and it
refuses calls whose scratch would not fit its static buffer.  This file is
collected last so that a run stopping at the first failure has run the rest."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def he():
    from paper_2403_11166_gb300 import he
    return he


def _share(shape, seed):
    g = torch.Generator(device="cpu").manual_seed(seed)
    return torch.randint(0, 1 << 41, shape, generator=g, dtype=torch.int64).cuda()


def test_noalloc_equals_encrypt_share_twice(he):
    ctx = he.Context(13, 3, 60)
    sk = ctx.keygen(9)
    conv = he.Plan(ctx, he.Layer(he.CONV, 8, 4, 4, 16, 16, 3, 1), he.ROLE_FWD, None)
    wgrad = he.Plan(ctx, he.Layer(he.FC, 16, 40, 12), he.ROLE_WGRAD, None)
    calls = [(conv, he.OPERAND_INPUT, _share((8, 4, 16, 16), 1), 11),
             (wgrad, he.OPERAND_KERNEL, _share((16, 12), 2), 12)]
    outs = []
    for plan, operand, share, seed in calls:          # two allocation-free calls in a row
        count = plan.sizes.ct_in if operand == he.OPERAND_INPUT else plan.sizes.pt
        ct = plan.new_ct(count)
        he.encrypt_share_noalloc(ctx, sk, plan, operand, share, seed, ct)
        outs.append(ct)
    torch.cuda.synchronize()
    for (plan, operand, share, seed), got in zip(calls, outs):
        count = plan.sizes.ct_in if operand == he.OPERAND_INPUT else plan.sizes.pt
        want = plan.new_ct(count)
        ws = plan.new_ws(plan.sizes.ws_encrypt)
        he.encrypt_share(ctx, sk, plan, operand, share, seed, want, ws)
        torch.cuda.synchronize()
        assert torch.equal(got, want)


def test_noalloc_at_exact_capacity(he):
    """1024 ciphertexts x 8192 coefficients fill the 8 MiB scratch exactly: the
    call is accepted and equals encrypt_share."""
    ctx = he.Context(13, 3, 60)
    sk = ctx.keygen(10)
    plan = he.Plan(ctx, he.Layer(he.FC, 1024, 16, 16), he.ROLE_FWD, (1, 16, 16, 1, 1, 1, 1))
    assert plan.sizes.ct_in * 8192 == 8 << 20
    share = _share((1024, 16), 4)
    got = plan.new_ct(plan.sizes.ct_in)
    he.encrypt_share_noalloc(ctx, sk, plan, he.OPERAND_INPUT, share, 21, got)
    want = plan.new_ct(plan.sizes.ct_in)
    he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, share, 21, want, plan.new_ws(plan.sizes.ws_encrypt))
    torch.cuda.synchronize()
    assert torch.equal(got, want)


def test_noalloc_rejects_oversized_call(he):
    ctx = he.Context(13, 3, 60)
    sk = ctx.keygen(9)
    # 1100 ciphertexts x 8192 coefficients = 9 MB of errors > the 8 MiB buffer
    plan = he.Plan(ctx, he.Layer(he.FC, 1100, 16, 16), he.ROLE_FWD, (1, 16, 16, 1, 1, 1, 1))
    assert plan.sizes.ct_in == 1100
    ct = torch.zeros((1100, 2, 3, 8192), dtype=torch.int64, device="cuda")
    with pytest.raises(he.PencilError) as e:
        he.encrypt_share_noalloc(ctx, sk, plan, he.OPERAND_INPUT, _share((1100, 16), 3), 1, ct)
    assert e.value.code == -4
    assert int(ct.abs().sum()) == 0
