"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI, compare."""
import numpy as np

from paper_0906_1887_gb300 import synth


def run_engine(packed, n, c, t, bits, engine, n_dumps=1, accumulate=False, vis_init=None, tuning=None,
               operands=None):
    import torch
    from paper_0906_1887_gb300 import corr
    plan = corr.Plan(n, c, t, bits)
    if tuning is not None:
        plan.set_tuning(*tuning)
    if operands is not None:
        plan.set_operands(*operands)
    dev = torch.device("cuda:0")
    x = torch.from_numpy(np.ascontiguousarray(packed).view(np.uint8).reshape(-1)).to(dev)
    vis = plan.empty_vis(n_dumps, dev)
    if vis_init is not None:
        vis.copy_(torch.from_numpy(vis_init))
    else:
        vis.fill_(-7)  # garbage the overwrite path must replace
    ws = plan.empty_workspace(engine, n_dumps, dev)
    plan.run(x, vis, ws, accumulate=accumulate, engine=engine, n_dumps=n_dumps)
    torch.cuda.synchronize()
    assert plan.check_device() == 0
    out = vis.cpu().numpy()
    plan.close()
    return out


def normwise_error(v, ref, n):
    """max |V - V64| / sqrt(V64_ii V64_jj) over channels and pairs (float error metric)."""
    iu, ju = np.triu_indices(n)
    auto_idx = [i * n - i * (i - 1) // 2 for i in range(n)]
    autos = ref[..., auto_idx, 0]                      # [..., N]
    scale = np.sqrt(np.maximum(autos[..., iu] * autos[..., ju], 1e-300))
    err = np.abs((v[..., 0] - ref[..., 0]) + 1j * (v[..., 1] - ref[..., 1]))
    return float((err / scale).max())


def check_bf16x3(got, samples, n, c, t, chans=None):
    """Hold every element of a BF16x3 result to the per-element error bound of the split
    products (oracle/precision.py: what BF16x3 drops, plus fp32 accumulation over the dump).
    The bound sits several times below the error of the variants that drop a correction
    product, so a kernel computing one of those fails here.  ``got`` holds the selected
    channels only.  Returns (normwise error against float64, largest error / bound)."""
    from oracle import precision
    bound, ex = precision.bf16x3_bound(samples, n, c, t, chans)
    g = np.asarray(got, np.float64)
    err = np.hypot(g[..., 0] - ex[..., 0], g[..., 1] - ex[..., 1])
    ratio = float((err / np.maximum(bound, 1e-300)).max())
    assert ratio <= 1.0, f"BF16x3 error exceeds its bound by a factor {ratio:.3g}"
    return normwise_error(g, ex, n), ratio


def int_case(seed, n, c, t, bits, lo=None, hi=None):
    if lo is None:
        lo, hi = (-8, 7) if bits == 4 else (-128, 127)
    re, im = synth.uniform_ints(seed, t, c, n, lo, hi)
    return synth.pack(re, im, bits)
