"""What the trained refinement gains over the plain method, in bf16 and in
its FP8 (E4M3) inference form.

Leave-one-camera-out renders of synthetic scenes on the nine-camera arc
(1/4 scale, 320x180, depth noise and dropouts as in the 1280x720 workload):
the network is trained on six scenes and evaluated on two unseen scenes,
against the held-out cameras' own frames."""
import numpy as np
import pytest

import synthetic as S
from fvv_helpers import lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def loo_data():
    F = lib()
    from paper_2007_00558_gb300 import refine_train as RT
    cams = S.rig_arc(9, 90.0, 1.5, 320, 180, 250.0)
    loo = RT.LooRig(cams, [0.0, 0.0, 0.0])
    try:
        def scene(seed):
            rgb, dep = S.frames_for(S.scene_random_objects(seed), cams, noise_seed=seed + 7)
            return loo.samples(rgb, dep)
        train = RT.concat([scene(s) for s in range(100, 106)])
        test = RT.concat([scene(s) for s in (200, 201)])
    finally:
        loo.close()
    return F, RT, cams, train, test


def test_refinement_improves_psnr_on_unseen_scenes(loo_data):
    F, RT, cams, train, test = loo_data
    net = F.fvv_create(F.rig(cams[:1], [0.0, 0.0, 0.0]))
    try:
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
        F.fvv_destroy(net)


def test_fp8_twin_of_the_wide_network(loo_data):
    """Widths 48/96/192 trained in bf16, then quantised to E4M3 (scales from
    a bf16 pass over training samples): the FP8 twin keeps the gain."""
    F, RT, cams, train, test = loo_data
    net = F.fvv_create(F.rig(cams[:1], [0.0, 0.0, 0.0]))
    try:
        F.fvv_refine_init(net, F.fvv_refine_default_cfg(seed=2, widths=(48, 96, 192)))
        RT.train(net, train, steps=600, batch=8, crop=128, lr=2e-3)
        bf = RT.evaluate(net, test)
        RT.quantize(net, train, n=8)
        assert F.fvv_refine_get_precision(net)[0] == F.FVV_PREC_E4M3
        q = RT.evaluate(net, test)
        print("48/96/192 LOO PSNR plain %.2f dB, bf16 %.2f dB, e4m3 %.2f dB" % (
            bf["psnr_plain"], bf["psnr_refined"], q["psnr_refined"]))
        assert bf["psnr_refined"] >= bf["psnr_plain"] + 0.3
        assert q["psnr_refined"] >= bf["psnr_refined"] - 0.3
        assert q["psnr_refined"] >= q["psnr_plain"] + 0.3
    finally:
        F.fvv_destroy(net)
