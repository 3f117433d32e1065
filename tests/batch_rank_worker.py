"""One rank of the two-rank batch test (run under torch.distributed.run, gloo,
every rank on cuda:0): decompose this rank's shard of the mixed batch with
truss_decompose_batch, gather every rank's outputs on rank 0 and save them."""
import os
import sys

import numpy as np
import torch
import torch.distributed as dist

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import graphgen  # noqa: E402
from paper_1205_6693_gb300 import truss as T  # noqa: E402
from paper_1205_6693_gb300.shard import shard_range  # noqa: E402


def main():
    graphs, out = int(sys.argv[1]), sys.argv[2]
    dist.init_process_group("gloo")
    rank, ws = dist.get_rank(), dist.get_world_size()
    g0, g1 = shard_range(graphs, rank, ws)
    ns, off, src, dst = graphgen.batch(g1 - g0, first=g0)
    dev = torch.device("cuda:0")
    s, d = torch.from_numpy(src).to(dev), torch.from_numpy(dst).to(dev)
    sup, tr = torch.empty_like(s), torch.empty_like(s)
    kmax = torch.empty(len(ns), dtype=torch.int32, device=dev)
    ctx = T.Context(0)
    ctx.decompose_batch(ns, off, s, d, sup, tr, kmax)
    torch.cuda.synchronize()
    ctx.close()
    mine = (g0, g1, off, sup.cpu().numpy(), tr.cpu().numpy(), kmax.cpu().numpy())
    parts = [None] * ws
    dist.all_gather_object(parts, mine)
    if rank == 0:
        np.save(out, np.array(parts, dtype=object), allow_pickle=True)
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
