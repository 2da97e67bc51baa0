"""Shared helpers of the GPU parity tests: build both sides from one seeded scene dict and compare
per-path results where the two followed the same branch (identical branch signatures)."""
import numpy as np

# Tolerances of the parity contract: per path / pixel relative error <= 1e-4 where the GPU (FP32)
# and the oracle (FP64) took the same branches, >= 99.9% of pixels agreeing.  The absolute floor
# (1e-6 of the image's largest value) only covers terms that are zero up to FP32 rounding.
RTOL = 1e-4
ATOL_REL = 1e-6
MIN_PIXEL_AGREEMENT = 0.999


def paths_close(g, o, scale):
    return np.all(np.abs(g - o) <= RTOL * np.abs(o) + ATOL_REL * scale, axis=-1)


def compare_with_oracle(gpu_L, gpu_sig, or_L, or_sig, spp, label=""):
    """gpu_L, or_L: (N_p, 3); sigs: (N_p,) uint32.  Returns a dict of agreement statistics and
    asserts the contract."""
    gpu_L = np.asarray(gpu_L, np.float64)
    gsig = np.asarray(gpu_sig).astype(np.uint32)
    osig = np.asarray(or_sig).astype(np.uint32)
    scale = max(1e-12, float(np.abs(or_L).max()))
    same = gsig == osig
    close = paths_close(gpu_L, or_L, scale)
    bad_same = same & ~close
    n_pix = gpu_L.shape[0] // spp
    pix_same = same.reshape(n_pix, spp).all(1)
    gp = gpu_L.reshape(n_pix, spp, 3).sum(1) / spp
    op = or_L.reshape(n_pix, spp, 3).sum(1) / spp
    pix_close = paths_close(gp, op, scale)
    agree = pix_same & pix_close
    res = {"paths": gpu_L.shape[0], "same_branch": float(same.mean()), "bad_same_branch": int(bad_same.sum()),
           "pixel_agreement": float(agree.mean())}
    if bad_same.any():
        i = np.flatnonzero(bad_same)[:5]
        res["examples"] = [(int(k), gpu_L[k].tolist(), or_L[k].tolist()) for k in i]
    assert res["bad_same_branch"] <= max(0, int(1e-5 * gpu_L.shape[0])), (label, res)
    assert res["pixel_agreement"] >= MIN_PIXEL_AGREEMENT, (label, res)
    return res
