"""Serving with continuous batching: jobs submitted while others run are admitted
as slots and device memory free up, advance together in batched launches, and end
with the same fields as when run alone (within the FP32 parity bound)."""
import time

import numpy as np
import pytest

from paper_1803_01756_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_01756_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def job_set(n, seed):
    u = inputs.uniform01(5 * n, seed).reshape(n, 5)
    jobs = []
    for k in range(n):
        nx, ny = int(48 + 300 * u[k, 0]), int(10 + 50 * u[k, 1])
        p = inputs.base_params(Gw=-1.2 + 0.1 * u[k, 2], u_period=float(300 + int(900 * u[k, 3])))
        steps = int(40 + 160 * u[k, 4])
        jobs.append((nx, ny, p, steps, inputs.noisy_density(nx, ny, inputs.RHO_V_086, 0.01, seed + k)))
    return jobs


def alone(job, storage=0):
    from paper_1803_01756_gb300.lattice import Lattice
    nx, ny, p, steps, rho0 = job
    lat = Lattice(nx, ny, p, kernel=2, storage=storage)
    lat.write_fields(rho0)
    lat.step(steps)
    out = lat.read_fields()
    lat.close()
    return out


# A job in the mix runs in the batched kernel, alone in the single-lattice kernel; the
# two compute the same update, so each job's fields must agree within the FP32 parity
# bound in either storage (measured on GB300: bitwise equal in FP32, BF16 and FP16).
SAME_BOUNDS = {0: {"rho": 1e-5, "u": 1e-5, "T": 1e-5},
               1: {"rho": 1e-5, "u": 1e-5, "T": 1e-5}}


def assert_same(got, ref, storage=0):
    rho, ux, uy, T = got
    rr, rux, ruy, rT = ref
    b = SAME_BOUNDS[storage]
    err = {"rho": np.abs(rho - rr).max() / np.abs(rr).max(),
           "u": np.hypot(ux - rux, uy - ruy).max() / max(np.hypot(rux, ruy).max(), 1e-3),
           "T": np.abs(T - rT).max() / np.abs(rT).max()}
    assert all(err[k] <= b[k] for k in b), err
    return err


@pytest.mark.parametrize("storage", [0, 1], ids=["f32", "bf16"])
def test_jobs_in_the_mix_equal_jobs_alone(storage):
    """Both storages: FP32, and BF16, the storage the serving workload runs."""
    from paper_1803_01756_gb300.lattice import JOB_DONE, Server
    jobs = job_set(9, seed=70)
    srv = Server(hbm_budget=1 << 34, max_active=8, chunk_steps=24)
    ids = []
    for k, (nx, ny, p, steps, rho0) in enumerate(jobs):
        ids.append(srv.submit(nx, ny, p, steps, rho0, storage=storage))
        if k % 3 == 2:
            time.sleep(0.05)  # later jobs arrive while earlier ones run
    for jid in ids:
        assert srv.wait(jid, 300) == JOB_DONE
    st = srv.stats()
    assert st["completed"] == len(jobs) and st["failed"] == 0
    for jid, job in zip(ids, jobs):
        state, fields, latency = srv.poll(jid, fields=True)
        assert state == JOB_DONE and latency > 0
        assert_same(fields, alone(job, storage), storage)
    srv.close()


def test_admission_respects_the_hbm_budget():
    from paper_1803_01756_gb300.lattice import JOB_DONE, Server
    jobs = job_set(6, seed=90)
    # room for about two of these jobs at a time
    budget = 2 * max(2 * 9 * ((nx + 31) // 32 * 32) * ny * 4 + 7 * ((nx + 31) // 32 * 32) * ny * 4
                     + nx * ny * 8 for nx, ny, *_ in jobs) + 100_000
    srv = Server(hbm_budget=budget, max_active=8, chunk_steps=16)
    ids = [srv.submit(nx, ny, p, steps, rho0) for nx, ny, p, steps, rho0 in jobs]
    for jid in ids:
        assert srv.wait(jid, 300) == JOB_DONE
    st = srv.stats()
    assert st["peak_bytes"] <= budget
    assert st["completed"] == len(jobs)
    srv.close()


def test_oversized_job_is_refused():
    from paper_1803_01756_gb300.lattice import LbmError, Server
    srv = Server(hbm_budget=1 << 20)
    with pytest.raises(LbmError) as ei:
        srv.submit(4096, 512, inputs.base_params(), 10)
    assert ei.value.code == -6
    srv.close()


def test_unstable_job_fails_alone_and_others_finish():
    from paper_1803_01756_gb300.lattice import JOB_DONE, Server
    jobs = job_set(3, seed=110)
    srv = Server(hbm_budget=1 << 34, max_active=8, chunk_steps=50)
    good = [srv.submit(nx, ny, p, steps, rho0) for nx, ny, p, steps, rho0 in jobs]
    bad_p = inputs.base_params(x_bc=0, **{"lambda": 40.0})
    bad = srv.submit(16, 8, bad_p, 400, inputs.noisy_density(16, 8, inputs.RHO_V_086, 0.01, 2))
    assert srv.wait(bad, 300) == -4
    for jid, job in zip(good, jobs):
        assert srv.wait(jid, 300) == JOB_DONE
        assert_same(srv.poll(jid, fields=True)[1], alone(job))
    srv.close()


def test_wait_times_out_and_destroy_cancels():
    from paper_1803_01756_gb300.lattice import Server
    srv = Server(hbm_budget=1 << 34, max_active=1, chunk_steps=50)
    jid = srv.submit(2048, 256, inputs.base_params(), 200000)
    assert srv.wait(jid, 0.05) == -5
    srv.close()
