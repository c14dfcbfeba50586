"""Host-side patch tables of the fused explicit step (no GPU). The tables come from the library's
own builder (the one a context uses); every property is recomputed here from the exported mesh
alone: the Morton runs and the greedy cut rule (64 cells, 640 hanging-table entries), the slot
lists and hanging tables of each patch, the swizzled shared-memory positions, the numbering by
decreasing work and the ownership of every dof. Meshes: the 64-instance batch configuration's
(Q2, a refinement ball, 278,581 dofs, 24,848 hanging nodes: the cap cuts patches), the ribbed
part's first layer at level 3 (Q2, trees masked out, inactive cells above the layer) and a small
Q1 mesh with nested refinement and an inactive top layer."""
import numpy as np
import pytest

from paper_2302_05164_gb300 import inputs as I
from paper_2302_05164_gb300 import pbf

CELLS, MAX_HENT = 64, 640


def swizzle(j):
    j = np.asarray(j, np.int64)
    return j ^ ((j >> 5) & 31)


def morton(anchor):
    key = np.zeros(len(anchor), np.uint64)
    for b in range(21):
        for a in range(3):
            key |= ((anchor[:, a].astype(np.uint64) >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + a)
    return key


def q1_mesh():
    regions = [I.uniform_region(1), (I.BALL, (0.4e-3, 0.25e-3, 0.2e-3), (0, 0, 0), 150e-6, 3)]
    return I.mesh_desc((8, 4, 2), (125e-6,) * 3, 1, 3, regions, active_top_z=0.2e-3, powder_z0=0.15e-3,
                       powder_z1=0.2e-3)


MESHES = {"c4": I.c4_mesh, "c5_level3": lambda: I.c5_mesh(level=3), "q1_inactive_layer": q1_mesh}


@pytest.fixture(scope="module", params=sorted(MESHES))
def mesh_tables(request):
    m = pbf.Mesh(MESHES[request.param]())
    mt, st, info = m.tables(), pbf.pbf_mesh_step_tables(m.h), m.info()
    m.close()
    assert len(st["ptr"]) > 0 and info["n_hanging"] > 0
    return mt, st, dict(info, name=request.param)


def patch_rows(mt, cells):
    """Rows referenced by the cells (sorted), the dofs they list with the rows' masters (sorted),
    and the hanging-table entries."""
    cd = mt["cell_dofs"][cells].ravel()
    rows = np.unique(-1 - cd[cd < 0])
    cp, ci = mt["con_ptr"], mt["con_idx"]
    masters = [ci[cp[r]:cp[r + 1]] for r in rows]
    dofs = np.unique(np.concatenate([cd[cd >= 0]] + masters)) if len(cd) else cd
    hent = int(sum(cp[r + 1] - cp[r] for r in rows))
    return rows, dofs, hent


def test_patches_are_morton_runs_cut_by_the_greedy_rule(mesh_tables):
    mt, st, info = mesh_tables
    nc = info["n_active"]
    act = mt["leaves"][:, 4] == 1
    assert act.sum() == nc
    key = morton(mt["leaves"][act][:, :3])
    assert len(np.unique(key)) == nc
    rank = np.empty(nc, np.int64)
    rank[np.argsort(key, kind="stable")] = np.arange(nc)
    cell = st["cell"]
    lens = (cell >= 0).sum(1)
    assert st["cells_per_patch"] == CELLS and cell.shape[1] == CELLS
    for q in range(len(cell)):  # lanes filled from 0, then -1
        assert (cell[q, :lens[q]] >= 0).all() and (cell[q, lens[q]:] == -1).all()
    used = np.concatenate([cell[q, :lens[q]] for q in range(len(cell))])
    assert np.array_equal(np.sort(used), np.arange(nc))  # every active cell in exactly one lane
    # each patch is a run of consecutive cells in the global Morton order, in lane order
    first = np.array([rank[cell[q, 0]] for q in range(len(cell))])
    for q in range(len(cell)):
        assert np.array_equal(rank[cell[q, :lens[q]]], first[q] + np.arange(lens[q]))
    runs = np.argsort(first)
    assert first[runs[0]] == 0 and np.array_equal(first[runs[1:]], first[runs[:-1]] + lens[runs[:-1]])
    # cut rule: a run ends when it is full or when the next cell's new rows would exceed the cap
    by_rank = np.argsort(rank)
    cp = mt["con_ptr"]
    short = 0
    for i, q in enumerate(runs):
        rows, _, hent = patch_rows(mt, cell[q, :lens[q]])
        assert hent <= MAX_HENT or lens[q] == 1
        if i + 1 == len(runs) or lens[q] == CELLS:
            continue
        short += 1
        nxt = mt["cell_dofs"][by_rank[first[q] + lens[q]]]
        new = np.setdiff1d(np.unique(-1 - nxt[nxt < 0]), rows)
        assert hent + int(sum(cp[r + 1] - cp[r] for r in new)) > MAX_HENT, q
    if info["name"] == "c4":
        assert short > 50  # the cap does cut patches on this mesh


def test_slot_lists_hanging_tables_and_positions(mesh_tables):
    mt, st, info = mesh_tables
    nd, npc = info["n_dofs"], info["nodes_per_cell"]
    cell, ptr, cnt, slot = st["cell"], st["ptr"], st["cnt"], st["slot"]
    lens = (cell >= 0).sum(1)
    cp, ci, cw = mt["con_ptr"], mt["con_idx"], mt["con_w"]
    at, hat, works = 0, 0, []
    for q in range(len(cell)):
        cells = cell[q, :lens[q]]
        rows, dofs, hent = patch_rows(mt, cells)
        nfree, nu = len(dofs), len(dofs) + len(rows)
        assert tuple(cnt[q]) == (nfree, nu, hat, hat + hent)
        assert ptr[q] == at  # concatenated in the numbering, each list padded to a multiple of 4
        s = slot[at:at + nu]
        assert np.array_equal(s[:nfree] & 0x7FFFFFFF, dofs)
        assert (slot[at + nu:at + (nu + 3) // 4 * 4] == 0).all()
        start = 0
        for j, r in enumerate(rows):
            n = cp[r + 1] - cp[r]
            assert s[nfree + j] == (start << 5) | n
            e = slice(hat + start, hat + start + n)
            assert np.array_equal(st["hloc"][e], swizzle(np.searchsorted(dofs, ci[cp[r]:cp[r + 1]])))
            assert np.array_equal(st["hw"][e], cw[cp[r]:cp[r + 1]].astype(np.float32))
            start += n
        # each lane's node: the swizzled index of its key (a dof, or nd + its hanging row)
        cd = mt["cell_dofs"][cells]
        idx = np.where(cd >= 0, np.searchsorted(dofs, np.maximum(cd, 0)), nfree + np.searchsorted(rows, -1 - cd))
        assert np.array_equal(st["loc"][q][:, :lens[q]], swizzle(idx).T)
        assert (st["loc"][q][:, lens[q]:] == 0).all()
        works.append(nu + 2 * hent)
        at += (nu + 3) // 4 * 4
        hat += hent
    assert at == len(slot) and hat == len(st["hloc"]) and nd > 0
    assert st["max_slots"] == max(cnt[:, 1]) and st["max_hent"] == max(cnt[:, 3] - cnt[:, 2])
    assert st["loc"].max() < 65536 and st["loc"].shape[1] == npc
    # numbered by decreasing work; equal work keeps the Morton order of the runs
    works = np.array(works)
    assert (np.diff(works) <= 0).all()
    rank_first = np.array([cell[q, 0] for q in range(len(cell))])
    key = morton(mt["leaves"][mt["leaves"][:, 4] == 1][:, :3])
    for q in np.nonzero(np.diff(works) == 0)[0]:
        assert key[rank_first[q]] < key[rank_first[q + 1]]


def test_every_dof_is_owned_by_the_first_patch_that_lists_it(mesh_tables):
    mt, st, info = mesh_tables
    nd = info["n_dofs"]
    owner = np.full(nd, -1)
    first = np.full(nd, -1)
    for q in range(len(st["ptr"])):
        nfree = st["cnt"][q, 0]
        s = st["slot"][st["ptr"][q]:st["ptr"][q] + nfree]
        d = s & 0x7FFFFFFF
        new = d[first[d] < 0]
        first[new] = q
        own = d[s < 0]  # bit 31 set
        assert (owner[own] == -1).all()
        owner[own] = q
    assert (owner >= 0).all()
    assert np.array_equal(owner, first)


def test_sizes_only_call_and_mismatched_sizes():
    m = pbf.Mesh(I.c1_mesh())
    L = pbf.lib()
    t = pbf.StepTables()
    assert L.pbf_mesh_step_tables(m.h, pbf.C.byref(t)) == 0
    assert (t.n_patches, t.n_hent, t.cells_per_patch, t.max_hent) == (512, 0, 64, 0)
    assert t.n_slots == 512 * 128 and t.max_slots == 125  # 125 dofs of a 4 x 4 x 4 block of Q1 cells
    buf = np.zeros(10, np.int32)
    t.n_patches, t.ptr = 10, buf.ctypes.data
    assert L.pbf_mesh_step_tables(m.h, pbf.C.byref(t)) == 1 and (buf == 0).all()
    assert L.pbf_mesh_step_tables(None, pbf.C.byref(t)) == 1
    assert L.pbf_mesh_step_tables(m.h, None) == 1
    m.close()
