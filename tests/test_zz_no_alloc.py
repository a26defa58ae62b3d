"""The allocation-free network forward against the regular one.

pnp_mlp_forward_noalloc serves callers that may not allocate device memory: it keeps
weights and activations in a fixed device array inside the library instead of a
context.  This file sorts last so that a run stopping at its first failure has run
every other test before it; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2301_05985_gb300 import workloads as W

from gpu_common import lib, torch_cuda

pytestmark = pytest.mark.gpu

TOL = 1e-2  # the network forward tolerance of the parity tests (BF16 operands)


def test_noalloc_forward_matches_context_forward_twice():
    pnp = lib()
    torch = torch_cuda()
    mesh = pnp.Mesh(W.uniform_octants(3, 2))
    ctx = pnp.Context(mesh, pnp.default_params(eps=0.05, dt=0.01), torch.cuda.current_stream().cuda_stream)
    ctx.mlp_init(seed=3)
    rng = np.random.default_rng(11)
    params = (rng.normal(size=pnp.PNP_MLP_PARAMS) * 0.08).astype(np.float32)
    ctx.mlp_set_weights(params)
    stream = torch.cuda.current_stream().cuda_stream
    dparams = torch.from_numpy(params).cuda()
    for B in (1000, pnp.PNP_NOALLOC_MAX_ROWS):
        X = torch.from_numpy(rng.normal(size=(B, 216)).astype(np.float32)).cuda()
        ref = torch.zeros((B, 3), dtype=torch.float32, device="cuda")
        ctx.mlp_forward(X, ref)
        ref = ref.cpu().numpy()
        Ys = [torch.full((B, 3), float("nan"), dtype=torch.float32, device="cuda") for _ in range(2)]
        pnp.mlp_forward_noalloc(dparams, X, Ys[0], stream)  # loads the array if not yet resident
        torch.cuda.synchronize()
        Ys[0].fill_(float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for Y in Ys:  # the shared scratch keeps the previous call's contents
            pnp.mlp_forward_noalloc(dparams, X, Y, stream)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0  # nothing was allocated on the device
        for Y in Ys:
            Y = Y.cpu().numpy()
            assert np.all(np.isfinite(Y))
            assert np.linalg.norm(Y - ref) <= TOL * np.linalg.norm(ref)
    # more rows than the fixed scratch holds: rejected with a clear error
    X = torch.zeros((pnp.PNP_NOALLOC_MAX_ROWS + 1, 216), dtype=torch.float32, device="cuda")
    Y = torch.zeros((pnp.PNP_NOALLOC_MAX_ROWS + 1, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(pnp.PnpError) as e:
        pnp.mlp_forward_noalloc(dparams, X, Y, stream)
    assert e.value.code == pnp.PNP_ERR_ARG and "scratch" in str(e.value)
    ctx.close()
    mesh.close()
