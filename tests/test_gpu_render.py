"""The image energies on the GPU (cloth_image_energy) against the oracle: rendered image,
silhouette, E = E_p + 0.5 E_s and dE/dx of a perturbed 4x4 sheet against the frame of
another perturbation (FP64)."""
import numpy as np
import pytest

from test_render_host import scene

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("seed,W,H", [(1, 24, 20), (2, 24, 20), (3, 96, 80)])
def test_image_energy_matches_oracle(seed, W, H):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import softras as S
    from paper_2203_11938_gb300 import sim

    x, tris, tri, uv, tex, cam, image, mask = scene(seed, W, H)
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")  # noqa: E731
    E, g, img, sil = sim.image_energy(cu(x), tris, cu(uv), cu(tex), cam, cu(image), cu(mask), want_grad=True,
                                      want_render=True)
    torch.cuda.synchronize()
    img_o, A_o = S.render(x, tri, uv, tex, cam, image.shape[1], image.shape[0])
    np.testing.assert_allclose(img.cpu().numpy(), img_o.numpy(), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(sil.cpu().numpy(), A_o.numpy(), rtol=1e-10, atol=1e-12)
    E_o, g_o = S.energy_and_grad(np.stack([x, x]), tri, uv, tex, cam, [None, image], [None, mask])
    assert float(E[0]) == pytest.approx(E_o, rel=1e-10)
    np.testing.assert_allclose(g.cpu().numpy(), g_o[1], rtol=1e-7, atol=1e-9 * np.abs(g_o[1]).max())
