"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and the oracle on the
same seeded inputs, and compare."""
import numpy as np
import torch

import oracle
from workloads import scenes

TOL_RGB = 2e-4      # absolute, per RGB / alpha channel
TOL_GRAD = 1e-3     # relative L2 per gradient array


def to_dev(scene, device="cuda"):
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(device)  # noqa: E731
    return f(scene.means), f(scene.quats), f(scene.scales), f(scene.opacities), f(scene.rgb)


def params(Q=None, eps1=1e-4, k_max=2 ** 31 - 1, background=(0.0, 0.0, 0.0), t_near=0.0, sort_key=0, eps2=None):
    from paper_2501_19196_gb300 import RenderParams
    return RenderParams(Q=scenes.default_Q() if Q is None else Q, eps1=eps1, t_near=t_near,
                        background=tuple(background), k_max=k_max, sort_key=sort_key, eps2=eps2)


def gpu_render(scene, cams, prm, tune=None, renderer=None, keep=False):
    from paper_2501_19196_gb300 import Renderer
    r = renderer or Renderer(tune=tune, Q_box=max(prm.Q, scenes.default_Q()))
    dev = to_dev(scene)
    r.build(*dev)
    rgb, alpha, depth = r.render(cams, prm)
    torch.cuda.synchronize()
    r.check_device()
    out = {"rgb": rgb.cpu().numpy().astype(np.float64), "alpha": alpha.cpu().numpy().astype(np.float64),
           "depth": depth.cpu().numpy().astype(np.float64)}
    if keep:
        return out, r, dev
    r.close()
    return out


def pixel_index(cams, cam, px, py):
    base = np.concatenate([[0], np.cumsum(cams.n_pixels())[:-1]])
    return base[cam] + py.astype(np.int64) * cams.width[cam].astype(np.int64) + px


def oracle_pixels(scene, cams, cam, px, py, prm, dl_rgb=None, dl_alpha=None, dl_depth=None):
    return oracle.render(scene, cams, cam, px, py, prm.Q, prm.eps1, prm.k_max, prm.background, prm.t_near,
                         dl_rgb=dl_rgb, dl_alpha=dl_alpha, sort_key=prm.sort_key, dl_depth=dl_depth,
                         eps2=prm.eps2)


# Largest fraction of pixels that the oracle may exclude from parity (IMPACT flag: an FP32
# decision that FP64 could take the other way changes the pixel by more than 1e-4).  The
# workloads' samples stay at or below it; tests with a different figure state why.
MAX_MASKED = 0.001


def compare_image(gpu, ora, idx, tol=TOL_RGB, max_masked=MAX_MASKED, label=""):
    """Element-wise parity on pixels whose value is unique at the tolerance (oracle's IMPACT
    flag clear).  Returns (max rgb/alpha error, masked fraction)."""
    ok = (ora["mask"] & oracle.AMB_IMPACT) == 0
    masked = 1.0 - ok.mean()
    e_rgb = np.abs(gpu["rgb"][idx][ok] - ora["rgb"][ok]).max(initial=0.0)
    e_a = np.abs(gpu["alpha"][idx][ok] - ora["alpha"][ok]).max(initial=0.0)
    e_d = (np.abs(gpu["depth"][idx][ok] - ora["depth"][ok]) / np.maximum(1.0, ora["depth"][ok])).max(initial=0.0)
    m = ora["mask"]
    print(f"[parity] {label}: pixels {len(m)} max|d rgb| {e_rgb:.3e} max|d alpha| {e_a:.3e} depth rel {e_d:.3e} "
          f"masked {masked:.4f} (boundary {np.mean(m & oracle.IMP_BOUNDARY != 0):.4f}, "
          f"tie {np.mean(m & oracle.IMP_TIE != 0):.4f}, eps1 {np.mean(m & oracle.IMP_EPS1 != 0):.4f}); "
          f"decision-flagged {np.mean(m & oracle.AMB_DECISION != 0):.4f}")
    assert e_rgb <= tol and e_a <= tol, f"{label}: rgb err {e_rgb}, alpha err {e_a}"
    assert e_d <= 1e-3, f"{label}: depth rel err {e_d}"
    assert masked <= max_masked, f"{label}: masked fraction {masked}"
    return max(e_rgb, e_a), masked


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
