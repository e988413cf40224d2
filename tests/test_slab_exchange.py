"""The transpose-free slab decomposition of Sec. 2.2 on CPU ranks: the strided
exchange against the paper's own 16-point, 2-process example, and a full
distributed r2c + c2r over gloo (world sizes 2 and 4) against the single-process
transform.  The library itself runs on one GPU (one slab per device, replicas
only); these tests pin the layout the sharded form would use."""
import os
import socket

import numpy as np
import pytest

import synth
from tests import slab_sim

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "slab_exchange_4x4.txt")


def _golden():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        r, sent, held = line.split()
        rows[int(r)] = ([int(v) for v in sent.split(",")], [int(v) for v in held.split(",")])
    return rows


def test_worked_example_of_the_strided_exchange():
    """Sec. 2.2: P0 selects [3, 4, 7, 8] and P1 [9, 10, 13, 14] of the 4 x 4
    array 1..16; after the exchange each holds its n1/p columns of every row,
    n0 outermost, with no local transpose."""
    a = np.arange(1, 17).reshape(4, 4)
    p = 2
    local = [a[0:2], a[2:4]]
    gold = _golden()
    held = {r: slab_sim.place_received([slab_sim.send_block(local[q], r, p) for q in range(p)], 2, 2, ())
            for r in range(p)}
    for r in range(p):
        assert list(slab_sim.send_block(local[r], 1 - r, p)) == gold[r][0]
        assert list(held[r].reshape(-1)) == gold[r][1]
        # held is n0 x (n1/p): row j0 at stride n1/p, the paper's strided n0 axis
        assert np.array_equal(held[r], a[:, 2 * r:2 * r + 2])
    # the inverse exchange restores each slab
    for r in range(p):
        back = slab_sim.place_returned([slab_sim.return_block(held[s], r, p) for s in range(p)], 2, 4, p, ())
        assert np.array_equal(back, local[r])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _to_t(z):
    import torch
    return torch.from_numpy(np.ascontiguousarray(z).view(np.float64).copy())


def _worker(rank, p, shape, port):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=p)
    try:
        n0, n1, n2 = shape
        n0p, b, H = n0 // p, n1 // p, n2 // 2 + 1
        x = synth.uniform_field(shape, seed=81)
        local = x[rank * n0p:(rank + 1) * n0p]
        # 1. 2D r2c of the rank's planes
        loc = np.fft.rfftn(local, axes=(1, 2))
        # 2. strided sends, contiguous receives
        reqs = [dist.isend(_to_t(slab_sim.send_block(loc, s, p)), dst=s) for s in range(p) if s != rank]
        blocks = []
        for q in range(p):
            if q == rank:
                blocks.append(slab_sim.send_block(loc, rank, p))
            else:
                t = torch.empty(2 * n0p * b * H, dtype=torch.float64)
                dist.recv(t, src=q)
                blocks.append(t.numpy().view(np.complex128))
        for r in reqs:
            r.wait()
        held = slab_sim.place_received(blocks, n0p, b, (H,))
        # 3. the n0 axis, in place at its stride (b*H)
        held = np.fft.fft(held, axis=0)
        ref = np.fft.rfftn(x)[:, rank * b:(rank + 1) * b, :]
        assert np.linalg.norm(held - ref) <= 1e-12 * np.linalg.norm(ref)
        # inverse in reverse order: n0, exchange back, 2D c2r (unnormalised)
        back = np.fft.ifft(held, axis=0) * n0
        reqs = [dist.isend(_to_t(slab_sim.return_block(back, q, p)), dst=q) for q in range(p) if q != rank]
        blocks = []
        for s in range(p):
            if s == rank:
                blocks.append(slab_sim.return_block(back, rank, p))
            else:
                t = torch.empty(2 * n0p * b * H, dtype=torch.float64)
                dist.recv(t, src=s)
                blocks.append(t.numpy().view(np.complex128))
        for r in reqs:
            r.wait()
        planes = slab_sim.place_returned(blocks, n0p, n1, p, (H,))
        y = np.fft.irfftn(planes, s=(n1, n2), axes=(1, 2)) * (n1 * n2)
        assert np.linalg.norm(y - n0 * n1 * n2 * local) <= 1e-12 * n0 * n1 * n2 * np.linalg.norm(local)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("p,shape", [(2, (8, 8, 6)), (4, (8, 12, 10)), (4, (16, 8, 16))])
def test_distributed_slab_r2c_c2r_over_gloo(p, shape):
    torch = pytest.importorskip("torch")
    torch.multiprocessing.spawn(_worker, args=(p, shape, _free_port()), nprocs=p, join=True)
