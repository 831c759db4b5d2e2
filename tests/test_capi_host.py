"""CPU checks of the C-ABI library: it loads, exports every entry point that
include/sem.h declares, and its host-only numbering of order-p triangle nodes
(sem_mesh_nodes2d) agrees with the oracle's canonical numbering.  No call here
touches a GPU."""
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sem():
    import paper_2009_00705_gb300 as pkg
    from paper_2009_00705_gb300 import build as B
    B.build()
    pkg.lib()
    return pkg


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:sem_status|void|const char\*)\s+(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sem_setup", "sem_apply", "pmg_vcycle", "laplace_solve", "sem_teardown", "sem_last_error"):
        assert required in names


def test_no_entry_point_takes_a_posix_semaphore_name():
    # the CUDA runtime linked into the library calls the POSIX sem_* functions; an entry point of
    # the same name would capture those calls inside the library
    posix = {"sem_init", "sem_destroy", "sem_post", "sem_wait", "sem_trywait", "sem_timedwait", "sem_clockwait",
             "sem_open", "sem_close", "sem_unlink", "sem_getvalue"}
    assert not posix & set(declared_functions())


def test_library_exports_every_declared_symbol(sem):
    L = sem.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
    assert set(declared_functions()) == set(sem.EXPORTS)


def test_default_options(sem):
    o = sem.sem_default_options(6)
    assert [o.level_p[i] for i in range(o.nlevels)] == [6, 3, 1]
    o = sem.sem_default_options(4)
    assert [o.level_p[i] for i in range(o.nlevels)] == [4, 2, 1]
    assert o.k_cheb == 5 and o.nu1 == 1 and o.nu2 == 1 and o.rtol == 1e-8 and o.cheb_lo == 0.01
    assert o.cheb_hi == 1.05 and o.lanczos_steps == 30 and o.learned_tau == 0.5 and o.batch_mode == 0 and o.autotune == 1
    assert o.asm_overlap == 1 and o.smoother == 0
    assert o.coarse_rtol == 1e-2 and o.coarse_imax == 5000


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_host_numbering_matches_oracle(sem, p):
    from oracle.mesh import Level
    from oracle.refelem import RefTri
    for mesh in (W.config_slice2d(), W.box3d(5, 3, 2)):
        lev = Level(mesh, p)
        xy = sem.sem_mesh_nodes2d(mesh, p)
        assert xy.shape == (lev.N2, 2)
        tn = RefTri(p).nodes
        for b in range(mesh.tri.shape[0]):
            np.testing.assert_allclose(xy[lev.map2[b]], lev.tri_node_xy(b, tn), atol=1e-13)


def test_bad_mesh_is_rejected_without_gpu(sem):
    m = W.config_slice2d()
    m.tri = m.tri.copy()
    m.tri[0, 0] = 10**6
    with pytest.raises(sem.SemError) as e:
        sem.sem_mesh_nodes2d(m, 3)
    assert e.value.status == sem.SEM_EINVAL
    assert "out of range" in sem.sem_last_error()


def _c_struct_fields(name):
    src = open(os.path.join(ROOT, "include", "sem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", src).group(1)
    fields = []
    kw = {"const", "unsigned", "signed", "long", "short", "int", "double", "float", "char", "*"}
    for decl in body.split(";"):
        decl = re.sub(r"\[[^\]]*\]", "", decl).replace("*", " * ")
        toks = decl.split()
        if not toks:
            continue
        i = next(k for k, t in enumerate(toks) if t not in kw)
        fields += [n.strip() for n in " ".join(toks[i:]).split(",")]
    return fields


@pytest.mark.parametrize("cname,pyname", [("sem_options", "SemOptions"), ("sem_stats", "SemStats"),
                                           ("sem_mesh", "SemMesh")])
def test_ctypes_structs_mirror_the_header(sem, cname, pyname):
    # a field missing on the Python side would let the library write past the
    # ctypes buffer; names and order must match exactly
    assert [f for f, _ in getattr(sem, pyname)._fields_] == _c_struct_fields(cname)


def test_unknown_option_is_an_error(sem):
    with pytest.raises(TypeError):
        sem.sem_default_options(4, no_such_option=1)


@pytest.mark.parametrize("p", [1, 3, 6])
def test_host_blended_nodes_match_oracle(sem, p):
    # the library's curved-triangle map (host side) against the oracle's at the order-p nodes
    from oracle.mesh import Level, blended_xy
    from oracle.refelem import RefTri
    mesh = W.hull_tank(8)
    lev = Level(mesh, p)
    xy = sem.sem_mesh_nodes2d(mesh, p)
    tn = RefTri(p).nodes
    for b in np.flatnonzero((mesh.edge_arc[:, :, 2] > 0).any(1)):
        np.testing.assert_allclose(xy[lev.map2[b]], blended_xy(mesh, b, tn), atol=1e-13)
    straight = np.flatnonzero(~(mesh.edge_arc[:, :, 2] > 0).any(1))[:20]
    for b in straight:
        np.testing.assert_allclose(xy[lev.map2[b]], lev.tri_node_xy(b, tn), atol=1e-13)


def test_bad_arc_is_rejected_without_gpu(sem):
    m = W.hull_tank(8)
    m.edge_arc = m.edge_arc.copy()
    b, f = np.argwhere(m.edge_arc[:, :, 2] > 0)[0]
    m.edge_arc[b, f, 2] *= 1.1             # the vertices no longer lie on the circle
    with pytest.raises(sem.SemError) as e:
        sem.sem_setup(m, 2)
    assert e.value.status == sem.SEM_EINVAL and "circle" in sem.sem_last_error()


def test_bad_hull_fields_are_rejected_without_gpu(sem):
    # column heights outside 1..nlayers, non-finite interfaces, and the prism-only fields on a
    # 2D mesh are refused before any device work
    m = W.hull_tank(8)
    m.col_layers = m.col_layers.copy()
    m.col_layers[3] = m.nlayers + 1
    with pytest.raises(sem.SemError) as e:
        sem.sem_setup(m, 2)
    assert e.value.status == sem.SEM_EINVAL and "col_layers" in sem.sem_last_error()
    m = W.hull_tank(8)
    m.z_iface = m.z_iface.copy()
    m.z_iface[2, 1] = np.nan
    with pytest.raises(sem.SemError) as e:
        sem.sem_setup(m, 2)
    assert "z_iface" in sem.sem_last_error()
    s2 = W.config_slice2d()
    s2.col_layers = np.ones(s2.tri.shape[0], dtype=np.int32)
    with pytest.raises(sem.SemError) as e:
        sem.sem_setup(s2, 2)
    assert "prism meshes only" in sem.sem_last_error()
