"""The trained weights of the LB warm start (paper_1303_2470_gb300/surrogate_weights.npz)
match the network the library runs: every layer's weight and bias shapes, the output scales
and the training record (CPU only; the GPU tests run the network)."""
import json
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PATH = os.path.join(ROOT, "paper_1303_2470_gb300", "surrogate_weights.npz")


@pytest.mark.skipif(not os.path.exists(PATH), reason="surrogate weights not trained")
def test_weights_match_the_network():
    from paper_1303_2470_gb300 import surrogate     # the layer table; no library is loaded
    layers = surrogate.LAYERS
    z = np.load(PATH, allow_pickle=False)
    meta = json.loads(str(z["meta"]))
    n = 0
    for name, cin, cout, _ in layers:
        W, b = z[name + ".W"], z[name + ".b"]
        assert W.shape == (27, cin, cout) and W.dtype == np.float32 and np.all(np.isfinite(W))
        assert b.shape == (cout,) and np.all(np.isfinite(b))
        n += W.size + b.size
    assert n == meta["n_params"] == 2_351_120
    assert meta["s_u"] > 0 and meta["s_rho"] > 0 and meta["force"] == 1e-5
    hist = [v for _, v in meta["val_history"]]
    assert len(hist) >= 2 and hist[-1] < hist[0]          # the held-out loss fell while training
