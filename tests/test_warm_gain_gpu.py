"""What the trained warm-start predictor gains over the method without it.

The predictor is trained on the GPU, by the library's own kernels, on (image, latents)
pairs that the library's encoder produced.  On held-out images it then starts the same
1000-iteration schedule as plain overfitting, in two variants: with the mean trained
decoder, and with the plain method's own seeded decoder.  Both must reach the plain run's
final RD cost (within 1 %) well before the plain run does.  The second variant changes
only the starting latents, so its gain is the network's alone."""
from concurrent.futures import ThreadPoolExecutor

import pytest

from paper_2403_11651_gb300 import warm_bench

pytestmark = pytest.mark.gpu


def test_trained_predictor_reaches_plain_rd_sooner():
    a = warm_bench.parser().parse_args(["--train", "32", "--test", "2", "--size", "256",
                                        "--iters", "1000", "--ablate", "2"])
    with ThreadPoolExecutor(4) as pool:
        r = warm_bench.experiment(a, pool)
    first, last = r["predictor_loss_first_last_epoch"]
    assert last < first, (first, last)
    for img in r["per_image"]:
        warm = img["warm_iters_to_plain_final"]
        latents_only = img["latents_only_iters_to_plain_final"]
        assert warm is not None and warm <= 600, img
        assert latents_only is not None and latents_only <= 850, img
        assert img["warm_final"] < img["plain_final"] * 1.01, img
