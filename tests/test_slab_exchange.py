"""The rank-level halo exchange of the z-slab decomposition
(``slabs.exchange_halo``) over torch.distributed, on the CPU with gloo at
world sizes 2 and 3.  Each rank holds one slab in the state layout (38 planes
of nx*ny*nz_local values, halo planes included); a stand-in step does pure
pull streaming on the slab's own planes.  Streaming is a permutation of the
lattice, so after T steps with an exchange after each the slabs' planes must
equal the whole lattice with every population plane rolled T cells along
its e_i -- which holds only if every face value reached the right halo plane
of the right rank every step."""
import os
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

E = np.array([(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
              (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1),
              (1, 0, -1), (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)])


def _stream_slab(state, nx, ny, nzl):
    """Pull streaming of the slab's own planes z = 1 .. nzl-2 (x, y periodic),
    reading the halo planes across the z faces."""
    nxy = nx * ny
    src = state[:, :nzl * nxy].reshape(38, nzl, ny, nx).clone()
    out = state[:, :nzl * nxy].reshape(38, nzl, ny, nx)
    for q in range(38):
        ex, ey, ez = (int(v) for v in E[q % 19])
        rolled = torch.roll(src[q], shifts=(ey, ex), dims=(1, 2))
        out[q, 1:nzl - 1] = rolled[1 - ez:nzl - 1 - ez]


def _worker(rank, world, port, nx, ny, nz, T, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from paper_0912_2913_gb300.slabs import exchange_halo, slab_planes, split_z

    dist.init_process_group("gloo", rank=rank, world_size=world)
    G = np.random.default_rng(7).standard_normal((38, nz, ny, nx))
    z0, z1 = split_z(nz, world)[rank]
    nzl = z1 - z0 + 2
    S = (nzl * nx * ny + 63) // 64 * 64
    state = torch.full((38, S), float("nan"), dtype=torch.float64)
    state[:, :nzl * nx * ny] = torch.from_numpy(G[:, slab_planes(z0, z1, nz)].reshape(38, -1))
    for _ in range(T):
        _stream_slab(state, nx, ny, nzl)
        exchange_halo(state, nx, ny, nzl)
    mine = state[:, :nzl * nx * ny].reshape(38, nzl, ny, nx)[:, 1:-1].numpy()
    want = np.stack([np.roll(G[q], shift=(T * E[q % 19][2], T * E[q % 19][1], T * E[q % 19][0]), axis=(0, 1, 2))
                     for q in range(38)])[:, z0:z1]
    out[rank] = bool(np.array_equal(mine, want))
    dist.destroy_process_group()


@pytest.mark.parametrize("world,nz", [(2, 7), (3, 8)])
def test_exchange_halo_reproduces_whole_lattice_streaming(world, nz):
    port = 29600 + (os.getpid() + 17 * world) % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, 5, 4, nz, 6, out), nprocs=world, join=True)
        res = dict(out)
    assert res == {r: True for r in range(world)}


def test_exchange_halo_single_process_is_periodic():
    """Without a process group the slab is its own neighbour: the exchange
    closes the ring in z, as a whole periodic lattice."""
    sys.path.insert(0, ROOT)
    from paper_0912_2913_gb300.slabs import exchange_halo, slab_planes

    nx, ny, nz, T = 4, 3, 5, 7
    G = np.random.default_rng(8).standard_normal((38, nz, ny, nx))
    nzl = nz + 2
    state = torch.from_numpy(np.ascontiguousarray(G[:, slab_planes(0, nz, nz)].reshape(38, -1)))
    for _ in range(T):
        _stream_slab(state, nx, ny, nzl)
        exchange_halo(state, nx, ny, nzl)
    mine = state.reshape(38, nzl, ny, nx)[:, 1:-1].numpy()
    want = np.stack([np.roll(G[q], shift=(T * E[q % 19][2], T * E[q % 19][1], T * E[q % 19][0]), axis=(0, 1, 2))
                     for q in range(38)])
    assert np.array_equal(mine, want)
