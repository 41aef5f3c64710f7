"""Worker processes for the gloo tests of the host-side sharding (spawned)."""
import datetime
import os
import sys
import traceback

import numpy as np


def oracle_scorer(n_t=40, n_f=60, seed=3, tau_max=0.01):
    """score_fn(offset, count, k) backed by the FP64 oracle on a small seeded map."""
    import oracle
    from paper_1401_8060_b300 import HIT_DTYPE, synth
    sig = synth.sigma_powerlaw(40.0 + 0.5 * np.arange(n_f))
    y = synth.noise_map(n_t, n_f, sig, 17)
    om = oracle.OracleMap(y, sig, 40.0, 0.5, True)

    def score(off, cnt, k):
        snr = om.score_range(seed, off, cnt, tau_max, nthreads=1)
        vals, idx = oracle.topk(snr, off, k)
        h = np.zeros(k, dtype=HIT_DTYPE)
        for i, (v, g) in enumerate(zip(vals, idx)):
            f, tau = oracle.track_params(seed, int(g), n_f, tau_max)
            h[i]["snr"], h[i]["index"], h[i]["f"], h[i]["tau"] = v, g, f, tau
        return h
    return score


def run_rank(rank, world, port, n_tracks, k, fail_rank, q):
    try:
        sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
        import torch.distributed as dist
        from paper_1401_8060_b300 import search
        dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", world_size=world, rank=rank,
                                timeout=datetime.timedelta(seconds=20))
        if rank == fail_rank:
            raise RuntimeError("rank %d fails before its collective" % rank)
        hits = search.distributed_topk(oracle_scorer(), n_tracks, k)
        q.put((rank, "ok", hits.tobytes()))
        dist.destroy_process_group()
    except Exception as e:  # report to the parent; a failed peer shows up here on the others
        q.put((rank, "error", repr(e) + traceback.format_exc()[-300:]))
