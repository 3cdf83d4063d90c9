"""The learned cost model against the method without it (GPU): trained on the autotuner's own
measurements of random compound skeletons, its choices on unseen skeletons must come closer to the
exhaustive tuner's best than the default configuration and the paper's nearest-neighbour
derivation do. A small version of `python -m paper_1510_06585_gb300.costmodel`."""
import numpy as np
import pytest

from paper_1510_06585_gb300 import costmodel as C
from paper_1510_06585_gb300 import mrw as M

pytestmark = pytest.mark.gpu


def test_learned_choices_come_within_ten_percent_and_beat_nearest_neighbour():
    # 4000 training and 500 unseen random skeletons of up to 2^26 elements, every one of the 16
    # candidate configurations timed by the exhaustive tuner
    res, model, std = C.experiment(n_train=4000, n_test=500, max_log2=26, epochs=300, reps=3, log=None)
    learned, default, nn = res["learned"], res["default_config"], res["nearest_neighbour_kb"]
    print({k: res[k] for k in ("learned", "nearest_neighbour_kb", "default_config")})
    assert learned["mean"] <= 0.10, res  # the workload's target: within 10 % of the tuner's best
    assert learned["mean"] < nn["mean"], res  # the paper's derivation above 3 dimensions (Section 3.2)
    assert learned["mean"] < default["mean"] and learned["mean"] < res["random_config"]["mean"], res
    assert res["final_train_loss"] < 1.0, res


def test_installed_model_drives_execute_without_a_config():
    lib = M.load()
    lib.mrw_kb_clear()
    arena = C.Arena(20)
    feats, times, specs = C.collect(300, 77, max_log2=20, reps=1, arena=arena)
    model, std, _, _ = C.train(feats, times, epochs=40)
    spec = specs[0]
    tree = C.build_tree(spec)
    args = C.sample_args(arena, spec)
    cfgs = M.tune_candidates(tree, args)
    # the library feeds raw features: fold the standardisation into the first layer, then the
    # library's choice must be the argmin of the same forward pass on the raw features
    pred_std = C.predict(model, std, feats[:1])
    C.fold_standardization(model, std)
    model.install(cfgs)
    try:
        best, _ = M.tune(tree, args, M.MRW_TUNE_MODEL)
        raw = M.features(tree, args)[None, :]
        import torch
        y = torch.zeros(1, 16, device="cuda")
        model.forward(torch.from_numpy(raw.astype(np.float32)).cuda(), y)
        torch.cuda.synchronize()
        assert best.as_tuple() == cfgs[int(y.argmin())].as_tuple()
        assert lib.mrw_kb_size() == 1
        # folding changes the predictions only by bf16 rounding of the folded weights
        assert np.abs(y.cpu().numpy() - pred_std).max() <= 0.05 * np.abs(pred_std).max() + 1e-3
    finally:
        lib.mrw_tune_set_model(None, None, 0)
        lib.mrw_kb_clear()
