"""Every scoring path on small maps of each weighting and precision: the workload
of the debug-build test (tests/test_gpu_debug_bounds.py).  Run as a script
(python tests/_debug_worker.py out.npz, with STK_LIBRARY naming the library) it
saves the results; the test also calls run_all() in its own process."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _map(mode, n_t, n_f, seed):
    from paper_1401_8060_b300 import synth
    rng = np.random.default_rng(seed)
    if mode == "pixel":
        sig = rng.uniform(0.5, 2.0, (n_t, n_f)).astype(np.float32)
    elif mode == "freq":
        sig = synth.sigma_powerlaw(40.0 + 0.5 * np.arange(n_f), 1.2)
    else:
        sig = np.full(n_f, 1.3, np.float32)
    return synth.noise_map(n_t, n_f, sig, seed + 7), sig


def run_all():
    import torch
    import paper_1401_8060_b300 as stk
    from paper_1401_8060_b300 import _lib
    out = {"build_flags": np.array([_lib.lib().stk_build_flags()])}
    ctx = stk.Context(0)
    n_t, n_f, tau_max = 40, 300, 0.01
    rng = np.random.default_rng(5)
    f3 = rng.integers(0, n_f, (300, 3)).astype(np.int32)
    f3[:20] = np.array([0, n_f - 1, 0], np.int32)          # the band edges
    tau = rng.uniform(-tau_max, tau_max, 300)
    fc = rng.uniform(0, n_f - 1, (64, 3)).astype(np.float32)
    tc = rng.uniform(-tau_max, tau_max, 64).astype(np.float32)
    cases = [(mode, fp16, paper) for mode in ("const", "freq", "pixel") for fp16 in (False, True)
             for paper in ((False, True) if (mode == "pixel" and not fp16) else (False,))]
    for mode, fp16, paper in cases:
        tag = f"{mode}_fp16{int(fp16)}_paper{int(paper)}"
        y, sig = _map(mode, n_t, n_f, 11)
        m = ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), 40.0, 0.5, paper_mode=paper,
                         fp16=fp16)
        ctx.set_tracks(20_000, 3, 5, tau_max)
        for kernel in (1, 2):
            ctx.set_option(_lib.STK_OPT_KERNEL, kernel)
            out[f"{tag}_all_k{kernel}"] = ctx.score_all(m).cpu().numpy()
            h = ctx.score(m, 16)
            out[f"{tag}_hits_k{kernel}"] = np.stack([h["snr"], h["index"].astype(np.float64)])
        ctx.set_option(_lib.STK_OPT_KERNEL, 0)
        out[f"{tag}_explicit"] = ctx.score_explicit(m, torch.from_numpy(f3).cuda(),
                                                    torch.from_numpy(tau).cuda()).cpu().numpy()
        ctx.set_template_shape(True, 5)
        ctx.set_tracks(5000, 4, 0, tau_max)
        out[f"{tag}_general"] = ctx.score_all(m).cpu().numpy()
        ctx.set_template_shape(False)
        fct, tct = torch.from_numpy(fc).cuda(), torch.from_numpy(tc).cuda()
        out[f"{tag}_interp"] = ctx.interp_forward(m, fct, tct).cpu().numpy()
        gf, gt = ctx.interp_adjoint(m, fct, tct, torch.ones(64, device="cuda"))
        out[f"{tag}_adjoint"] = np.concatenate([gf.cpu().numpy().ravel(), gt.cpu().numpy()])
        fr, tr, _ = ctx.refine(m, fct, tct, tau_max, steps=5)
        out[f"{tag}_refine"] = np.concatenate([fr.cpu().numpy().ravel(), tr.cpu().numpy()])
        fp, tp, sp, wp = ctx.polish(m, f3[:32], tau[:32], tau_max, alt_f3=fr[:32], alt_tau=tr[:32], moves=3)
        out[f"{tag}_polish"] = np.concatenate([fp.cpu().numpy().ravel().astype(np.float64), tp.cpu().numpy(),
                                               sp.cpu().numpy()])
        ctx.sync()
        m.close()
    maps = []
    for i, (nt, nf) in enumerate([(30, 200), (55, 310), (41, 257)]):
        y, sig = _map("freq", nt, nf, 20 + i)
        maps.append(ctx.load_map(torch.from_numpy(y).cuda(), torch.from_numpy(sig).cuda(), 40.0, 0.5))
    b = stk.Batch(ctx, maps, [30_000, 20_000, 25_000], [7, 8, 9], [0, 0, 0], tau_max)
    hb = b.score(4).reshape(-1)
    out["batch"] = np.stack([hb["snr"], hb["index"].astype(np.float64)])
    b.close()
    for mm in maps:
        mm.close()
    ctx.sync()
    ctx.close()
    return out


if __name__ == "__main__":
    res = run_all()
    np.savez(sys.argv[1], **res)
    print("ok", len(res))
