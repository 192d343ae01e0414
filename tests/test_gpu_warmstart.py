"""The learned warm start gains over the FBP start: a network trained by the
library's own BF16 kernels on (FBP, OS-LALM) pairs of a small fan-beam scan
family gives held-out initial images closer to the converged PWLS image, and
OS-LALM started from them stays closer over the first iterations."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_network_start_is_closer_to_converged_image():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1402_4381_gb300 import build, warmstart as WS
    build.build()
    res = WS.experiment(n_train=96, n_test=8, target_iters=100, epochs=40, batch=8, lr=1e-3, nx=128, nviews=246,
                        ns=222, M=6, ref_schedule=((6, 30), (2, 50)), n_eval_iter=10, ref_block=200,
                        ref_max_iters=6000, log=lambda s: None)
    fbp = np.array(res["configured"]["fbp_init"]["rmsd_hu_mean_by_iteration"])
    cnn = np.array(res["configured"]["cnn_init"]["rmsd_hu_mean_by_iteration"])
    loss = res["train"]["loss_by_epoch"]
    assert np.mean(loss[-5:]) < 0.7 * loss[0]
    assert cnn[0] < 0.95 * fbp[0]
    assert np.all(cnn[:6] < fbp[:6])
    assert cnn.sum() < fbp.sum()
    # every x* converges, and the subset-reduction route reaches 1 HU from both
    # starts on every scan
    assert res["reference"]["converged"] == 8, res["reference"]
    for start in ("fbp_init", "cnn_init"):
        assert res["route"][start]["thresholds"]["1"]["reached"] == 8, res["route"][start]
