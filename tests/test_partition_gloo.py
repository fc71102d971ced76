"""The multi-GPU split of a ragged batch (independent images, no collective
in the data path): every rank computes the same partition of the 64-image
workload by pixel count, every image lands on exactly one rank, the loads
are balanced, and each rank's slice has the same per-image plan
(bs_batch_plan, host arithmetic) as in the one-rank batch.  Two gloo ranks
on CPU."""

import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2503_16424_gb300 import bs, synth
    from paper_2503_16424_gb300.batch import partition_images
    W = synth.BATCH_WORKLOAD
    layout = synth.batch_layout(W["seed"], W["n_images"], W["side"], W["aspect"], W["curves"])
    weights = [e["W"] * e["H"] for e in layout]
    parts = partition_images(weights, world)
    mine = parts[rank]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    cfg = bs.SampleCfg()
    images = [bs.BatchImage(e["W"], e["H"], e["n_open"], e["n_closed"], cfg) for e in layout]
    # the slice's totals are the sums of its images' one-image plans, which
    # are the images' entries of the whole batch
    whole = bs.batch_sizes(images, 16, 1 << 20)
    sub = bs.batch_sizes([images[i] for i in mine], 16, 1 << 20)
    each = [bs.batch_sizes([images[i]], 16, 1 << 20) for i in mine]
    ok_sum = all(sub[k] == sum(e[k] for e in each) for k in ("n_open", "n_closed", "n_gauss", "n_pixels", "n_tiles"))
    dist.barrier()
    out.put((rank, parts, gathered, mine, ok_sum, whole, [weights[i] for i in mine]))
    dist.destroy_process_group()


def test_two_ranks_split_the_batch_exactly_once_and_balanced():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, parts0, gath0, mine0, ok0, whole, w0), (r1, parts1, gath1, mine1, ok1, _, w1) = res
    assert parts0 == parts1                       # every rank computes the same split
    assert gath0 == gath1 == [mine0, mine1]
    allidx = sorted(mine0 + mine1)
    assert allidx == list(range(64))              # each image exactly once
    assert ok0 and ok1
    l0, l1 = sum(w0), sum(w1)
    assert abs(l0 - l1) <= max(w0 + w1)           # LPT: within one image of even
    assert l0 + l1 == whole["n_pixels"]


def test_partition_edge_cases():
    from paper_2503_16424_gb300.batch import partition_images
    assert partition_images([5, 5, 5], 1) == [[0, 1, 2]]
    assert partition_images([3, 1], 4) == [[0], [1], [], []]
    assert partition_images([], 2) == [[], []]
    w = [7, 3, 3, 2, 2, 2]
    p = partition_images(w, 2)      # 7 | 3, 3 | +2 right | +2 left | +2 right
    assert p == [[0, 4], [1, 2, 3, 5]]
    assert sorted(sum(w[i] for i in q) for q in p) == [9, 10]
