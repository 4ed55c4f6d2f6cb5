"""The allocation-free energy entry point against the CPU oracle (needs a GPU).

cem_state_energy_noalloc serves callers that cannot allocate device memory
(an application whose device memory all belongs to its own fixed arena, or a
monitor that must not call cudaMalloc / cudaFree, which synchronise the
device, while other streams run).  It keeps its scratch in one fixed device
array shared by every call.  Here calls in a row, on meshes of different
sizes (each smaller than the one before, so stale rows of the earlier call
stay in the scratch), must give the oracle's strain energy of the state
(orc_strain_energy: ES-FEM edge strains, A/4 of each edge point per element)
and its kinetic energy 1/2 sum m |v|^2 with the oracle's lumped masses, to
1e-12 relative (the same FP64 arithmetic, partial sums grouped differently),
and the KE and SE the handle API records at step 0 for the same state.  The
last case is a 3 x 2 mesh with a hole at the boundary, where the lumped
mass of a node and the edges that are smoothed depend on which neighbours
are missing.

This file is named so that pytest collects it last."""
import numpy as np
import pytest

from paper_2509_01827_gb300 import inputs

REL = 1e-12


@pytest.fixture(scope="module")
def _built():
    from paper_2509_01827_gb300 import build
    build.build()


def _case(nx, ny, active, plane_strain, seed):
    p = inputs.Problem(name=f"noalloc_{nx}x{ny}", nx=nx, ny=ny, hx=1e-3, hy=1e-3,
                       active=active, energy_every=1)
    p.material.gc_uniform = 1e30
    p.material.plane_strain = plane_strain
    rng = np.random.default_rng(seed)
    n = p.n_nodes
    u = rng.standard_normal(2 * n) * 1e-6
    v = rng.standard_normal(2 * n) * 1e-2
    return p, u, v


def _handle_energy(p, u, v):
    """KE and SE of the step-0 energy record of the handle API."""
    from paper_2509_01827_gb300.cem import CEM_FP64, Solver
    s = Solver(p, precision=CEM_FP64)
    n = p.n_nodes
    s.set_state(ux=u[:n], uy=u[n:], vx=v[:n], vy=v[n:])
    s.step(1)
    e = s.energy()
    s.close()
    return e["KE"][0], e["SE"][0]


def _oracle_energy(p, u, v):
    """The oracle's SE of u and 1/2 sum m |v|^2 with its lumped masses."""
    from oracle.oracle import from_problem
    o = from_problem(p)
    n = p.n_nodes
    o.set_state(ux=u[:n], uy=u[n:], vx=v[:n], vy=v[n:])
    m = o.nodes()["m"]
    ke = 0.5 * float(np.sum(m * (v[:n] ** 2 + v[n:] ** 2)))
    return ke, o.strain_energy()


def _noalloc_energy(p, u, v):
    import torch
    from paper_2509_01827_gb300 import cem
    dev = torch.device("cuda", 0)
    ud = torch.from_numpy(u).to(dev)
    vd = torch.from_numpy(v).to(dev)
    act = None if p.active is None else torch.from_numpy(np.asarray(p.active, np.uint8)).to(dev)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(0)[0]
    m = p.material
    cem.cem_state_energy_noalloc(p.nx, p.ny, p.hx, p.hy, 0 if act is None else act.data_ptr(),
                                 m.E, m.nu, m.rho, m.plane_strain, ud.data_ptr(), vd.data_ptr(),
                                 out.data_ptr(), 0)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info(0)[0]
    ke, se = out.cpu().numpy()
    return ke, se, free0 - free1


@pytest.mark.gpu
def test_calls_in_a_row_match_the_oracle_and_the_handle_api(_built):
    import torch
    torch.cuda.init()
    edge_hole = np.ones(6, np.uint8)
    edge_hole[2] = 0                                                 # corner element out
    cases = [
        _case(40, 40, inputs.hole_mask(40, 0.04, 0.008), True, 11),  # plate with a hole
        _case(20, 13, None, False, 12),                              # fewer rows, plane stress
        _case(3, 2, edge_hole, True, 13),                            # hole at the boundary
    ]
    oracle = [_oracle_energy(*c) for c in cases]
    handle = [_handle_energy(*c) for c in cases]
    got = [_noalloc_energy(*c) for c in cases]  # calls in a row
    for (ke_o, se_o), (ke_h, se_h), (ke, se, grown) in zip(oracle, handle, got):
        assert ke_o > 0 and se_o > 0
        assert abs(ke - ke_o) <= REL * ke_o, (ke, ke_o)
        assert abs(se - se_o) <= REL * se_o, (se, se_o)
        assert abs(ke - ke_h) <= REL * ke_h, (ke, ke_h)
        assert abs(se - se_h) <= REL * se_h, (se, se_h)
    # later calls found the scratch already set up: device memory in use did
    # not grow during them
    assert got[1][2] == 0 and got[2][2] == 0


def test_rejects_meshes_beyond_the_scratch_limit(_built):
    """Size checks come before any device call, so this runs without a GPU."""
    from paper_2509_01827_gb300 import cem
    with pytest.raises(cem.CemError) as ei:
        cem.cem_state_energy_noalloc(4, 16385, 1e-3, 1e-3, 0, 32e9, 0.2, 2450.0, True, 1, 1, 1, 0)
    assert ei.value.code == cem.CEM_ERR_ARG
    assert "16384" in str(ei.value)
