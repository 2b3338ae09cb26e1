"""Shared helpers of the GPU tests: device buffers (torch) and matching
parameter blocks for the library and the oracle."""
import numpy as np


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("these tests need a CUDA GPU")
    return torch


def dev(a):
    torch = torch_cuda()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def lib_params(I, n, **kw):
    p = I.icd2s_default_params(n)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def orc_params(orc, lp):
    """The oracle's parameter block with the same values as the library's."""
    return orc.Params(z=lp.z, K=lp.K, m_min=lp.m_min, m_max=lp.m_max, m_init=lp.m_init or lp.m_max,
                      alpha=lp.alpha, c=lp.c, sweeps=lp.sweeps, T_max=lp.T_max, T_min=lp.T_min,
                      w1=lp.w1, w2=lp.w2, w3=lp.w3, mut_mode=lp.mut_mode, mut_rate=lp.mut_rate,
                      patience=lp.patience, max_iters=lp.max_iters, select_mode=lp.select_mode,
                      im_mode=lp.im_mode, ablation=lp.ablation, aspiration=lp.aspiration,
                      im_order=lp.im_order)
