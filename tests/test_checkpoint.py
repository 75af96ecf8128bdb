"""Checkpoint files of a chain (hqmc_checkpoint_write / hqmc_checkpoint_read): host
code only, so these run without a GPU.  Round trip bit for bit, header-only reads,
and every damaged file refused with HQMC_EIO."""
import os

import numpy as np
import pytest
import torch


@pytest.fixture(scope="module")
def hq():
    from paper_2508_16298_gb300 import build
    build.build()
    from paper_2508_16298_gb300 import hqmc
    return hqmc


def field():
    from paper_2508_16298_gb300 import inputs
    return torch.from_numpy(inputs.theta_hot(6, 10, 3))


def test_round_trip_is_bit_exact(hq, tmp_path):
    th = field()
    w = np.random.default_rng(1).standard_normal(3808).astype(np.float32)

    class FakeNet:
        def get_weights(self):
            return w

    path = str(tmp_path / "chain.ckp")
    hq.save_checkpoint(path, th, seed=42, traj_counter=17, dt=0.005, nsteps=20, solver="pmixed", trajectories=17,
                       accepted=13, J=1.25, K=1.0, noncompact=True, net=FakeNet())
    hdr, th2, w2 = hq.load_checkpoint(path)
    assert torch.equal(th, th2) and np.array_equal(w, w2)
    assert (hdr["L"], hdr["Ntau"], hdr["seed"], hdr["traj_counter"], hdr["nsteps"]) == (6, 10, 42, 17, 20)
    assert hdr["dt"] == 0.005 and hdr["J"] == 1.25 and hdr["K"] == 1.0 and hdr["action"] == hq.ACTION_NONCOMPACT
    assert hdr["solver"] == hq.SOLVER_PMIXED and (hdr["trajectories"], hdr["accepted"]) == (17, 13)
    assert hdr["n_weights"] == 3808 and hdr["version"] == 1


def test_damaged_files_are_refused(hq, tmp_path):
    th = field()
    path = str(tmp_path / "chain.ckp")
    hq.save_checkpoint(path, th, seed=1, traj_counter=2, dt=0.01, nsteps=10)
    raw = open(path, "rb").read()
    cases = {"flipped": raw[:200] + bytes([raw[200] ^ 1]) + raw[201:], "truncated": raw[:-9],
             "magic": b"X" + raw[1:]}
    for name, data in cases.items():
        bad = str(tmp_path / (name + ".ckp"))
        open(bad, "wb").write(data)
        with pytest.raises(hq.HQMCError) as e:
            hq.load_checkpoint(bad)
        assert e.value.status == hq.EIO, name
    with pytest.raises(hq.HQMCError) as e:
        hq.load_checkpoint(str(tmp_path / "missing.ckp"))
    assert e.value.status == hq.EIO
    with pytest.raises(hq.HQMCError) as e:  # odd L: not a lattice of this library
        hq.save_checkpoint(str(tmp_path / "odd.ckp"), torch.zeros((4, 5, 5, 2), dtype=torch.float64), seed=1,
                           traj_counter=0, dt=0.01, nsteps=1)
    assert e.value.status == hq.EINVAL
    assert not os.path.exists(str(tmp_path / "odd.ckp"))
