"""The device-built BVH (rg_mesh_create_gpu_bvh) against the host builder, the oracle
and the structural rules a traversal relies on: the host builder's node array bit for
bit with the same triangles in every leaf, counts bit-identical to the oracle's, every
triangle in exactly one leaf and inside the box of every node above it, depth within
the traversal stack, the same tree on every build, and the median split of ranges that
no bin split separates."""
import time

import numpy as np
import pytest
import torch

import synth
from oracle import mcrt
from paper_2511_04277_gb300 import api
from paper_2511_04277_gb300._native import RadgebError

pytestmark = pytest.mark.gpu


def check_bvh(mesh, m):
    """Structural validation of a mesh's BVH; returns its depth (root = 1)."""
    nodes, rec = mesh.bvh()
    nt = m.n_tris
    assert np.array_equal(np.sort(rec), np.arange(nt))               # the records are a permutation
    ints = nodes[:, 12:16].copy().view(np.int32)
    v = m.verts[m.tris]                                               # [nt, 3, 3]
    tlo, thi = v.min(axis=1), v.max(axis=1)
    covered = np.zeros(nt, np.int32)
    seen = np.zeros(len(nodes), np.int32)
    depth = 0
    inf = np.float32(np.inf)
    stack = [(0, 1, np.full(3, -inf), np.full(3, inf))]
    while stack:
        nd, d, alo, ahi = stack.pop()
        seen[nd] += 1
        depth = max(depth, d)
        for s in range(2):
            lo = np.array([nodes[nd, 4 * s], nodes[nd, 4 * s + 2], nodes[nd, 8 + 2 * s]])
            hi = np.array([nodes[nd, 4 * s + 1], nodes[nd, 4 * s + 3], nodes[nd, 9 + 2 * s]])
            clo, chi = np.maximum(alo, lo), np.minimum(ahi, hi)       # every box above must hold the triangles
            ref, cnt = ints[nd, s], ints[nd, 2 + s]
            if cnt > 0:
                assert cnt <= 4 and 0 <= ref and ref + cnt <= nt
                tri = rec[ref:ref + cnt]
                covered[ref:ref + cnt] += 1
                assert np.all(tlo[tri] >= clo) and np.all(thi[tri] <= chi), (nd, s)
            else:
                assert 0 < ref < len(nodes)
                stack.append((ref, d + 1, clo, chi))
    assert np.all(covered == 1)                                       # every record in exactly one leaf
    assert np.all(seen == 1)                                          # every node reached once
    assert depth == mesh.info()["bvh_depth"] and depth + 1 <= 64
    return depth


def same_tree(host, dev):
    """The device tree is the host tree: equal node arrays, the same triangles per leaf."""
    (nh, rh), (nd, rd) = host.bvh(), dev.bvh()
    assert np.array_equal(nh.view(np.uint32), nd.view(np.uint32))
    ints = nh[:, 12:16].copy().view(np.int32)
    for s in range(2):
        for ref, cnt in zip(ints[:, s], ints[:, 2 + s]):
            if cnt > 0:
                assert sorted(rh[ref:ref + cnt]) == sorted(rd[ref:ref + cnt])


def coincident(k=40):
    """k copies of one triangle in one face plus a square: no bin split separates the copies."""
    verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [2, 0, 1], [3, 0, 1], [3, 1, 1], [2, 1, 1]], np.float32)
    tris = [[0, 1, 2]] * k + [[3, 4, 5], [3, 5, 6]]
    return synth.meshes.Mesh(name="coincident", verts=verts, tris=np.array(tris, np.int32),
                             tri_face=np.array([0] * k + [1, 1], np.int32), n_faces=2,
                             patch_of_face=np.arange(2, dtype=np.int32), n_patches=2)


@pytest.mark.parametrize("name", ["plates16", "small_sat", "spacecraft", "coincident"])
def test_device_tree_is_the_host_tree(rg_ctx, name):
    m = {"plates16": lambda: synth.plates(16), "coincident": coincident}.get(name, getattr(synth, name, None))()
    t0 = time.perf_counter()
    host = api.Mesh.from_synth(rg_ctx, m, use_bvh=1)
    t1 = time.perf_counter()
    dev = api.Mesh.from_synth(rg_ctx, m, use_bvh=1, gpu_bvh=True)
    t2 = time.perf_counter()
    dh, dd = check_bvh(host, m), check_bvh(dev, m)
    ih, idv = host.info(), dev.info()
    print(f"{name}: {m.n_tris} triangles; host {1e3 * (t1 - t0):.1f} ms, device {1e3 * (t2 - t1):.1f} ms; "
          f"depth {dh}, {ih['bvh_nodes']} nodes, visits {ih['sah_visits']:.4f} / {idv['sah_visits']:.4f}")
    assert (dd, idv["bvh_nodes"], idv["refill"]) == (dh, ih["bvh_nodes"], ih["refill"])
    assert abs(idv["sah_visits"] - ih["sah_visits"]) <= 1e-5 * ih["sah_visits"]
    same_tree(host, dev)


def test_device_bvh_is_deterministic(rg_ctx):
    m = synth.spacecraft()
    a = api.Mesh.from_synth(rg_ctx, m, gpu_bvh=True).bvh()
    b = api.Mesh.from_synth(rg_ctx, m, gpu_bvh=True).bvh()
    assert np.array_equal(a[0].view(np.uint32), b[0].view(np.uint32)) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("schedule", [2, 3], ids=["lockstep", "refill"])
def test_counts_bit_exact_with_device_bvh(rg_ctx, schedule):
    m = synth.plates(16)
    rays = np.full(m.n_faces, 3000, np.int64)
    rays[5] = 0
    rays[77] = 65536 + 9
    mesh = api.Mesh.from_synth(rg_ctx, m, use_bvh=schedule, gpu_bvh=True)
    assert mesh.info()["refill"] == (schedule == 3)
    g = api.trace(rg_ctx, mesh, rays, 4).cpu().numpy()
    o = mcrt.trace_counts(m.verts, m.tris, m.tri_face, m.n_faces, rays, 4)
    assert np.array_equal(g, o)
    s2 = np.full(2 * m.n_faces, 500, np.int64)
    gs = api.trace_sided(rg_ctx, mesh, s2, 4).cpu().numpy()
    os_ = mcrt.trace_sided(m.verts, m.tris, m.tri_face, m.n_faces, s2, 4)
    assert np.array_equal(gs, os_)


@pytest.mark.parametrize("name,rows", [("small_sat", [0, 900, 2047]), ("spacecraft", [0, 5000, 10239])])
def test_device_bvh_rows_against_the_oracle(rg_ctx, name, rows):
    w = synth.workload(name, rays_scale=0.05)
    m = w["mesh"]
    dev = api.Mesh.from_synth(rg_ctx, m, gpu_bvh=True)
    host = api.Mesh.from_synth(rg_ctx, m)
    g = api.trace(rg_ctx, dev, w["rays"], w["seed"]).cpu().numpy()
    h = api.trace(rg_ctx, host, w["rays"], w["seed"]).cpu().numpy()
    assert np.array_equal(g, h)                                       # the two builders, every row
    o = mcrt.trace_counts(m.verts, m.tris, m.tri_face, m.n_faces, w["rays"], w["seed"], faces=rows)
    for r in rows:
        assert np.array_equal(g[r], o[r]), r


def test_small_meshes(rg_ctx):
    for n_sub in (2, 3, 5):                                          # 16, 36, 100 triangles
        m = synth.perpendicular_squares(n_sub)
        mesh = api.Mesh.from_synth(rg_ctx, m, use_bvh=1, gpu_bvh=True)
        check_bvh(mesh, m)
        same_tree(api.Mesh.from_synth(rg_ctx, m, use_bvh=1), mesh)
        rays = np.full(m.n_faces, 20000, np.int64)
        g = api.trace(rg_ctx, mesh, rays, 8).cpu().numpy()
        assert np.array_equal(g, mcrt.trace_counts(m.verts, m.tris, m.tri_face, m.n_faces, rays, 8, use_bvh=False))
    m = coincident()
    mesh = api.Mesh.from_synth(rg_ctx, m, use_bvh=1, gpu_bvh=True)
    rays = np.full(2, 20000, np.int64)
    g = api.trace(rg_ctx, mesh, rays, 8).cpu().numpy()
    assert np.array_equal(g, mcrt.trace_counts(m.verts, m.tris, m.tri_face, 2, rays, 8, use_bvh=False))
    cube = api.Mesh.from_synth(rg_ctx, synth.cube(), gpu_bvh=True)   # 12 triangles, -1: no BVH
    assert cube.info()["bvh_nodes"] == 0


def test_device_builder_refuses_bad_input(rg_ctx):
    m = synth.plates(4)
    v = m.verts.copy()
    v[3, 1] = np.nan
    with pytest.raises(RadgebError, match="RG_ERR_ARG"):
        api.Mesh(rg_ctx, v, m.tris, m.tri_face, m.n_faces, use_bvh=1, gpu_bvh=True)
    torch.cuda.synchronize()
