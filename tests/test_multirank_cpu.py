"""The N > 1 path of bench.py on CPU: two gloo ranks rendezvous on 127.0.0.1, pass the
barrier and agree on the slowest replica's time (replicas only: no data-path collective).
Each rank also runs an independent oracle two-site update on its own seed, as the GPU
replicas do with their own inputs, and the gathered energies differ by rank."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import numpy as np
    import torch
    import torch.distributed as dist

    import bench
    from oracle import bose_hubbard as bh
    from oracle import contract as oc
    from oracle import lanczos as olz
    from paper_1610_02244_gb300 import synth

    w, r, _ = bench.dist_setup()
    assert (w, r) == (ws, rank) and dist.get_backend() == "gloo"
    bench.barrier(w)
    tmax = bench.dist_max(float(rank + 1), w)
    # an independent replica: a small H_eff ground state on this rank's seed
    g = synth.rng(100 + rank)
    Le, Re = synth.hermitian_env(g, 6), synth.hermitian_env(g, 6)
    Ws, _, _ = bh.bh_mpo(4, 2, 1.0, 2.0)
    th = synth.complex_gaussian(g, (6, 3, 3, 6))
    E, *_ = olz.lanczos_ground(lambda x: oc.heff_apply(Le, Ws[1], Ws[2], Re, x), th)
    es = [torch.zeros(1, dtype=torch.float64) for _ in range(w)]
    dist.all_gather(es, torch.tensor([E], dtype=torch.float64))
    bench.barrier(w)
    out[rank] = (tmax, [float(e) for e in es], float(np.float64(E)))
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas():
    ws = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(ws, port, out), nprocs=ws, join=True,
                       start_method="spawn")
    assert out[0][0] == out[1][0] == 2.0           # max over ranks
    assert out[0][1] == out[1][1]                  # both see every replica's result
    assert out[0][2] != out[1][2]                  # replicas are independent problems
