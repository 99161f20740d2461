"""Pins of the oracle's Marching Cubes triangulation (R10: triangles from a cube-case analysis,
vertices at edge midpoints, Sec. 4.3).

A wrong face rule or a wrong loop direction breaks these: every case uses exactly its sign
changing edges; meshes of random sign fields (ambiguous faces included) whose boundary layer
is outside are closed and consistently oriented (every directed edge has exactly one reverse);
a sphere's mesh has Euler characteristic 2, outward normals and about the sphere's volume."""
import numpy as np

import oracle

EDGES = [(0, 1), (1, 2), (2, 3), (3, 0), (4, 5), (5, 6), (6, 7), (7, 4), (0, 4), (1, 5), (2, 6),
         (3, 7)]


def test_each_case_uses_exactly_its_crossing_edges():
    for c in range(256):
        t = oracle.tri_case(c)
        crossing = {j for j, (a, b) in enumerate(EDGES) if ((c >> a) & 1) != ((c >> b) & 1)}
        assert set(t.ravel().tolist()) == crossing, c
        assert len(t) <= 5
        for tri in t:
            assert len(set(tri.tolist())) == 3
    assert len(oracle.tri_case(0)) == 0 and len(oracle.tri_case(255)) == 0


def volume_from(F, s=0.01):
    """Oracle volume holding voxel values F[x, y, z] (weight 1) in blocks from the origin."""
    n = F.shape[0]
    nb = (n + 7) // 8
    keys, vals = [], []
    for bx in range(nb):
        for by in range(nb):
            for bz in range(nb):
                blk = np.ones((8, 8, 8))   # outside (positive) beyond the field
                sub = F[8 * bx:8 * bx + 8, 8 * by:8 * by + 8, 8 * bz:8 * bz + 8]
                blk[:sub.shape[0], :sub.shape[1], :sub.shape[2]] = sub
                keys.append((bx, by, bz))
                vals.append(blk.transpose(2, 1, 0).reshape(512))   # lx + 8 ly + 64 lz
    o = oracle.OracleVolume(s, 0.04, 64.0, 0.001, 0.0, 8, 8, 4.0, 4.0, 4.0, 4.0)
    keys = np.array(keys, np.int32)
    o.load(keys, np.array(vals), np.ones((len(keys), 512)))
    return o, keys


def mesh(o, keys):
    tris = o.triangles(keys)
    q = np.round(tris / 0.005).astype(np.int64)   # vertices on the half-voxel lattice
    return q


def directed_edges(q):
    e = {}
    for t in q:
        for a, b in ((0, 1), (1, 2), (2, 0)):
            k = (tuple(t[a]), tuple(t[b]))
            e[k] = e.get(k, 0) + 1
    return e


def test_random_fields_give_closed_oriented_meshes():
    rng = np.random.default_rng(0)
    for trial in range(6):
        n = 14
        F = np.where(rng.random((n, n, n)) < 0.45, -1.0, 1.0)
        F[0, :, :] = F[-1, :, :] = F[:, 0, :] = F[:, -1, :] = F[:, :, 0] = F[:, :, -1] = 1.0
        o, keys = volume_from(F)
        q = mesh(o, keys)
        assert len(q) > 100
        e = directed_edges(q)
        for (a, b), m in e.items():
            assert m == 1, "a directed edge used twice"
            assert e.get((b, a), 0) == 1, "an edge without its reverse"


def test_sphere_mesh_topology_volume_and_orientation():
    n, r = 24, 9.3
    g = np.arange(n) - 11.6
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    F = np.sqrt(X ** 2 + Y ** 2 + Z ** 2) - r
    o, keys = volume_from(F)
    q = mesh(o, keys)
    verts = {tuple(v) for t in q for v in t}
    und = {tuple(sorted(k)) for k in directed_edges(q)}
    assert len(verts) - len(und) + len(q) == 2   # Euler characteristic of a sphere
    P = q.astype(np.float64) * 0.5   # voxels
    vol = np.einsum("ij,ij->i", P[:, 0], np.cross(P[:, 1], P[:, 2])).sum() / 6.0
    assert vol > 0   # normals point to the outside (positive values)
    assert abs(vol - 4.0 / 3.0 * np.pi * r ** 3) < 0.06 * 4.0 / 3.0 * np.pi * r ** 3


def test_library_table_equals_the_oracle_derivation():
    """The two derivations (library host code, oracle) are written separately; the tables
    they produce must be identical, case by case and triangle by triangle."""
    from paper_1805_03709_b300 import build
    build.build()
    from paper_1805_03709_b300 import vbh as V
    n, e = V.vbh_mc_tri_table()
    for c in range(256):
        t = oracle.tri_case(c)
        assert n[c] == len(t), c
        np.testing.assert_array_equal(e[c, :3 * n[c]].reshape(-1, 3), t)
