"""Multi-GPU sweep path on one GPU: virtual ranks run one after another.

Sec. 8 of the paper: the DD sweep partitions by subdomains and only interface
data crosses between GPUs.  Each virtual rank sweeps its rectangle of
subdomains (hz_sweep_rect) into its own lambda buffer, packs the slots it
wrote for subdomains of other ranks (hz_lambda_gather, in the slot order of
partition.Partition's send plan), the buffers are handed over, and each rank
unpacks what it receives (hz_lambda_scatter).  The slots every rank owns, and
its subdomains' solutions, must equal one whole-problem hz_sweep bit for bit:
every subdomain runs the same kernel with the same arithmetic."""

import numpy as np
import pytest

from paper_2606_21695_gb300.partition import Partition
from workloads import configs

pytestmark = pytest.mark.gpu


def _rect(part, rank):
    bx, by = rank % part.px, rank // part.px
    return part.xe[bx], part.ye[by], part.xe[bx + 1] - part.xe[bx], part.ye[by + 1] - part.ye[by]


def _slots_dev(slots):
    import torch

    return torch.tensor(np.asarray(slots, dtype=np.int32).reshape(-1), dtype=torch.int32, device="cuda")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("world", [2, 3, 4])
def test_virtual_ranks_equal_single_sweep_bitwise(hz, precision, world):
    import torch

    from paper_2606_21695_gb300.api import Case

    wl = configs.Workload("part", (0.0, 1.0, 0.0, 1.0), 24, 18, 3, 4, 3, 11.0, "random", (0.4, 0.55), 0.06,
                          corr_len=0.3)  # 6 x 6 subdomains of 13 x 10 nodes
    case = Case(wl)
    prec = hz.HZ_FP64 if precision == "fp64" else hz.HZ_FP32_REFINE
    try:
        m_Sx, m_Sy = wl.nx // wl.sub_nx, wl.ny // wl.sub_ny
        nl = hz.hz_lambda_size(case.pr)
        NE = nl // (m_Sx * m_Sy * 4)
        nsub = (wl.sub_nx * wl.P + 1) * (wl.sub_ny * wl.P + 1)
        nt = hz.hz_problem_nt(case.pr)
        gen = torch.Generator(device="cuda").manual_seed(3)
        lam_in = torch.randn(2 * nl, dtype=torch.float64, device="cuda", generator=gen)
        rhs = torch.empty(2 * case.n, dtype=torch.float64, device="cuda")
        hz.hz_rhs(case.pr, rhs)
        ref_l = torch.zeros_like(lam_in)
        ref_u = torch.zeros(2 * m_Sx * m_Sy * nsub, dtype=torch.float64, device="cuda")
        hz.hz_sweep(case.pr, prec, nt, 3, 0.0, lam_in, ref_l, rhs, ref_u)

        part = Partition(m_Sx, m_Sy, world)
        outs, us = {}, {}
        for r in range(world):  # every rank's sweep, into its own buffers
            outs[r] = torch.full_like(lam_in, float("nan"))
            us[r] = torch.full_like(ref_u, float("nan"))
            hz.hz_sweep_rect(case.pr, prec, nt, 3, 0.0, _rect(part, r), lam_in, outs[r], rhs, us[r])
        sent = {}
        for r in range(world):  # pack the cut-interface slots per destination
            for dst, slots in part.send_plan(r).items():
                buf = torch.empty(2 * len(slots) * NE, dtype=torch.float64, device="cuda")
                hz.hz_lambda_gather(case.pr, _slots_dev(slots), len(slots), outs[r], buf)
                sent[(r, dst)] = buf
        for r in range(world):  # unpack what arrives
            for src, slots in part.recv_plan(r).items():
                hz.hz_lambda_scatter(case.pr, _slots_dev(slots), len(slots), sent[(src, r)], outs[r])
        torch.cuda.synchronize()
        ref_lc = ref_l.view(m_Sx * m_Sy, 4, NE, 2).cpu().numpy()
        ref_uc = ref_u.view(m_Sx * m_Sy, nsub, 2).cpu().numpy()
        seen = np.zeros(m_Sx * m_Sy, bool)
        for r in range(world):
            mine = part.subdomains(r)
            got_l = outs[r].view(m_Sx * m_Sy, 4, NE, 2).cpu().numpy()
            got_u = us[r].view(m_Sx * m_Sy, nsub, 2).cpu().numpy()
            assert np.array_equal(got_l[mine], ref_lc[mine]), r
            assert np.array_equal(got_u[mine], ref_uc[mine]), r
            seen[mine] = True
        assert seen.all()
    finally:
        case.close()


def test_sweep_rect_rejects_rectangles_outside_the_grid(hz):
    import torch

    from paper_2606_21695_gb300.api import Case

    case = Case(configs.scaled(configs.config1(), 16, 16, 4, 4, name="rect_bad"))
    try:
        nl = hz.hz_lambda_size(case.pr)
        a = torch.zeros(2 * nl, dtype=torch.float64, device="cuda")
        b = torch.zeros_like(a)
        nt = hz.hz_problem_nt(case.pr)
        for rect in [(0, 0, 5, 1), (3, 0, 2, 1), (0, -1, 1, 1), (0, 0, 0, 1)]:
            with pytest.raises(hz.HzError) as e:
                hz.hz_sweep_rect(case.pr, hz.HZ_FP64, nt, 1, 0.0, rect, a, b)
            assert e.value.status == hz.HZ_ERR_INVALID_ARG
    finally:
        case.close()


def test_lambda_slots_outside_the_vector_are_skipped(hz):
    import torch

    from paper_2606_21695_gb300.api import Case

    case = Case(configs.scaled(configs.config1(), 8, 8, 4, 4, name="slots_bad"))  # 2 x 2 subdomains
    try:
        nl = hz.hz_lambda_size(case.pr)
        NE = nl // (4 * 4)
        lam = torch.arange(2 * nl, dtype=torch.float64, device="cuda")
        slots = _slots_dev([(1, 2), (4, 0), (-1, 1), (3, 4), (2, 3)])  # 2nd-4th are outside
        buf = torch.full((2 * 5 * NE,), float("nan"), dtype=torch.float64, device="cuda")
        hz.hz_lambda_gather(case.pr, slots, 5, lam, buf)
        out = lam.clone()
        hz.hz_lambda_scatter(case.pr, slots, 5, buf * 0 - 1, out)
        torch.cuda.synchronize()
        b = buf.view(5, NE, 2).cpu().numpy()
        lv = lam.view(4, 4, NE, 2).cpu().numpy()
        assert np.array_equal(b[0], lv[1, 2]) and np.array_equal(b[4], lv[2, 3])
        assert not np.any(b[1:4])
        o = out.view(4, 4, NE, 2).cpu().numpy()
        changed = np.argwhere(np.any(o != lv, axis=(2, 3)))
        assert sorted(map(tuple, changed)) == [(1, 2), (2, 3)]
    finally:
        case.close()
