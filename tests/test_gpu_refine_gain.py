"""What the trained refinement gains over the plain method.

Leave-one-camera-out renders of synthetic scenes on the nine-camera arc
(1/4 scale, 320x180, depth noise and dropouts as in the 1280x720 workload):
the network is trained on six scenes and evaluated on two unseen scenes,
against the held-out cameras' own frames."""
import numpy as np
import pytest

import synthetic as S
from fvv_helpers import lib

pytestmark = pytest.mark.gpu


def test_refinement_improves_psnr_on_unseen_scenes():
    F = lib()
    from paper_2007_00558_gb300 import refine_train as RT
    cams = S.rig_arc(9, 90.0, 1.5, 320, 180, 250.0)
    loo = RT.LooRig(cams, [0.0, 0.0, 0.0])
    net = F.fvv_create(F.rig(cams[:1], [0.0, 0.0, 0.0]))
    try:
        def scene(seed):
            rgb, dep = S.frames_for(S.scene_random_objects(seed), cams, noise_seed=seed + 7)
            return loo.samples(rgb, dep)
        train = RT.concat([scene(s) for s in range(100, 106)])
        test = RT.concat([scene(s) for s in (200, 201)])
        F.fvv_refine_init(net, F.fvv_refine_default_cfg(seed=1))
        before = RT.evaluate(net, test)
        losses = RT.train(net, train, steps=600, batch=8, crop=128, lr=2e-3)
        after = RT.evaluate(net, test)
        print("LOO PSNR plain %.2f dB, untrained %.2f dB, trained %.2f dB (loss %.5f -> %.5f)" % (
            after["psnr_plain"], before["psnr_refined"], after["psnr_refined"],
            np.mean(losses[:20]), np.mean(losses[-20:])))
        assert np.mean(losses[-20:]) < np.mean(losses[:20])
        assert after["psnr_refined"] >= after["psnr_plain"] + 0.3
    finally:
        loo.close()
        F.fvv_destroy(net)
