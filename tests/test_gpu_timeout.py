"""The bounded waits of the tensor-core kernels, exercised on the GPU
without a fault: the test hook makes the tensor-core Gram issue no operand
loads, every wait runs out after its limit, the call reports FQ_ERR_TIMEOUT
through its status word, and the same context then computes a correct Gram."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_05464_gb300 import build as fqbuild
from paper_2509_05464_gb300 import fq

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fqbuild.build()
    fq.lib()


def test_tensor_core_wait_runs_out_and_reports_timeout():
    rng = np.random.default_rng(5)
    S = (rng.standard_normal((1000, 16)) + 1j * rng.standard_normal((1000, 16))).astype(np.complex64)
    Sd = torch.from_numpy(np.stack([S.real, S.imag], -1).astype(np.float32)).cuda()
    ws = fq.workspace(fq.fq_gram_workspace_size(1000, 16, fq.FQ_GRAM_BF16), torch.device("cuda"))
    lib = fq.lib()
    lib.fq_debug_set.argtypes = [fq._I32, fq._I32]
    assert lib.fq_debug_set(1, 1) == 0
    try:
        fq.fq_casorati_gram(Sd, gram_mode=fq.FQ_GRAM_BF16, ws=ws)
        with pytest.raises(fq.FqError) as e:
            fq.fq_clutter_status(ws)
        assert e.value.status == 6  # FQ_ERR_TIMEOUT
    finally:
        assert lib.fq_debug_set(1, 0) == 0
    # the context is still usable: a normal launch on the same workspace
    G = fq.fq_casorati_gram(Sd, gram_mode=fq.FQ_GRAM_BF16, ws=ws)
    fq.fq_clutter_status(ws)
    g = G.double().cpu().numpy()
    G = g[..., 0] + 1j * g[..., 1]
    Sq = torch.from_numpy(np.stack([S.real, S.imag], -1)).bfloat16().double().numpy()
    want = oracle.gram(Sq[..., 0] + 1j * Sq[..., 1])
    assert np.abs(G - want).max() <= 1e-5 * np.abs(want).max()
    assert lib.fq_debug_set(9, 1) == 1  # unknown setting
