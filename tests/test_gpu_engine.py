"""Persistent batched engine (GPU): parity with the one-trajectory-per-thread FP32 kernel and the
oracle, determinism under batching, the prefix stop rule, censoring and error paths."""
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle import mfpt, stats

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_1802_05065_gb300 as m
    return m


@pytest.fixture(scope="module")
def api():
    from paper_1802_05065_gb300 import api as _api
    return _api


def _engine(lib, **kw):
    kw.setdefault("chunk_steps", 4096)
    return lib.Engine(0, **kw)


def _run(eng, d, n, seed, **over):
    rid = eng.submit(lib_params(d, **over), n, seed)
    res = eng.wait(rid, 600.0)
    return rid, res


def lib_params(d, **over):
    import paper_1802_05065_gb300 as m
    return m.params_from(d, **over)


CONST_OVER = workloads.scaled(workloads.overdamped_sweep(n_traj=1)[11], max_steps=10**8)
CONST_UNDER = workloads.scaled(workloads.plain_constant_tilt(), D=0.05, precision="fp32",
                               max_steps=10**6, hist_hi=2000.0)


@pytest.mark.parametrize("d", [CONST_OVER, CONST_UNDER], ids=["overdamped", "underdamped"])
@pytest.mark.parametrize("T", [1, 2])
def test_engine_matches_plain_fp32_per_trajectory(lib, api, d, T):
    """Constant bias: the engine's lanes run the same single-precision arithmetic as the plain
    kernel, so every trajectory's escape step is identical, whatever lane ran it."""
    n, seed = 5000, 31
    with _engine(lib, traj_per_thread=T) as eng:
        rid, res = _run(eng, d, n, seed, keep_per_traj=1)
        e_steps = eng.per_traj_steps(rid, n)
    p_steps = api.run_plain(d, n, seed).cpu().numpy()
    assert (e_steps == p_steps).all()
    s = stats.summarize(oracle.params_from(d), e_steps)
    assert res.n_used == n and res.n_escaped == s.n_escaped
    assert math.isclose(res.mean, s.mean, rel_tol=1e-12)
    assert math.isclose(res.var, s.var, rel_tol=1e-9)


def test_engine_histogram_and_sums_exact(lib):
    d = workloads.scaled(CONST_UNDER, hist_bins=64, hist_lo=0.0, hist_hi=800.0)
    with _engine(lib) as eng:
        rid, res = _run(eng, d, 3000, 8, keep_per_traj=1)
        steps = eng.per_traj_steps(rid, 3000)
        h, u, o = eng.histogram(rid, 64)
    s = stats.summarize(oracle.params_from(d), steps)
    assert list(h) == list(s.hist) and u == s.under and o == s.over
    assert res.steps_total == sum(int(k) if k >= 0 else d["max_steps"] for k in steps)


def test_engine_statistics_vs_oracle(lib):
    """Underdamped constant tilt, FP32 engine vs FP64 oracle with independent seeds."""
    d = CONST_UNDER
    with _engine(lib) as eng:
        rid, res = _run(eng, d, 2**15, 101, keep_per_traj=1)
        g = eng.per_traj_steps(rid, 2**15)
    r = oracle.run(oracle.params_from(d), 202, 3000)
    p = oracle.params_from(d)
    sr = stats.summarize(p, r)
    assert stats.within_combined_se(res.mean, res.sem, sr.mean, sr.sem, 3.0)
    assert stats.ks_pvalue(stats.observables(p, g), stats.observables(p, r)) > 0.01


def test_engine_ramp_vs_oracle(lib):
    """Alg. 3 (switching bias) with a fast ramp: FP32 engine vs FP64 oracle."""
    d = workloads.ramp_sweep(n_traj=1, rates=(1e-4,))[0]
    with _engine(lib) as eng:
        rid, res = _run(eng, d, 2**14, 5, keep_per_traj=1)
        g = eng.per_traj_steps(rid, 2**14)
    r = oracle.run(oracle.params_from(d), 6, 1500)
    p = oracle.params_from(d)
    sr = stats.summarize(p, r)
    assert res.n_censored == 0 and sr.n_censored == 0
    assert stats.within_combined_se(res.mean, res.sem, sr.mean, sr.sem, 3.0)
    assert stats.ks_pvalue(stats.observables(p, g), stats.observables(p, r)) > 0.01


def test_batch_invariance(lib):
    """A request gives the same per-trajectory steps, histogram and sums alone and inside an
    uneven batch of requests of both models."""
    target = workloads.scaled(CONST_UNDER, hist_bins=50, hist_hi=1000.0)
    n, seed = 6000, 17
    with _engine(lib) as eng:
        rid, alone = _run(eng, target, n, seed, keep_per_traj=1)
        s_alone = eng.per_traj_steps(rid, n)
        h_alone = eng.histogram(rid, 50)
    mix = [(CONST_OVER, 20000, 1), (workloads.scaled(CONST_UNDER, D=0.08), 9000, 2),
           (workloads.ramp_sweep(n_traj=1, rates=(1e-3,))[0], 7000, 3)]
    with _engine(lib, chunk_steps=1024) as eng:
        others = [eng.submit(lib_params(d), k, s) for d, k, s in mix[:2]]
        rid = eng.submit(lib_params(target, keep_per_traj=1), n, seed)
        others.append(eng.submit(lib_params(mix[2][0]), mix[2][1], mix[2][2]))
        mixed = eng.wait(rid, 600.0)
        s_mix = eng.per_traj_steps(rid, n)
        h_mix = eng.histogram(rid, 50)
        for o in others:
            eng.wait(o, 600.0)
    assert (s_alone == s_mix).all()
    assert h_alone == h_mix
    assert (alone.mean, alone.var, alone.n_escaped) == (mixed.mean, mixed.var, mixed.n_escaped)


def test_stop_rule_prefix_matches_oracle_rule(lib):
    """The engine stops at the first whole-block prefix with relative SE <= target; the
    oracle's rule applied to the same escape steps keeps the same prefix."""
    d = workloads.scaled(CONST_OVER, stop_rse=0.02, stop_block=256)
    n = 2**16
    with _engine(lib) as eng:
        rid, res = _run(eng, d, n, 41, keep_per_traj=1)
        steps = eng.per_traj_steps(rid, n)
    assert res.n_used < n
    used = steps[: res.n_used]
    want = stats.stop_prefix(oracle.params_from(d), used, 0.02, 256)
    assert res.n_used == want
    s = stats.summarize(oracle.params_from(d), used)
    assert math.isclose(res.mean, s.mean, rel_tol=1e-12)
    assert res.sem <= 0.02 * res.mean


def test_censoring_and_budget(lib):
    """A tiny step budget censors every trajectory; a budget not a multiple of 4 censors at
    exactly max_steps (escape after the budget counts as censored)."""
    d = workloads.scaled(CONST_UNDER, max_steps=1001)
    with _engine(lib) as eng:
        rid, res = _run(eng, d, 4000, 3, keep_per_traj=1)
        steps = eng.per_traj_steps(rid, 4000)
    assert res.n_censored + res.n_escaped == 4000
    assert (steps[steps >= 0] <= 1001).all()
    d0 = workloads.scaled(CONST_UNDER, D=0.0)
    with _engine(lib) as eng:
        rid, res = _run(eng, workloads.scaled(d0, max_steps=5000), 700, 3)
    assert res.n_censored == 700 and math.isnan(res.mean)


def test_ragged_and_tiny_requests(lib, api):
    with _engine(lib) as eng:
        for n in (1, 31, 33, 4097):
            rid, res = _run(eng, CONST_OVER, n, 5, keep_per_traj=1)
            steps = eng.per_traj_steps(rid, n)
            assert res.n_used == n
            ref = api.run_plain(CONST_OVER, n, 5).cpu().numpy()
            assert (steps == ref).all()


def test_full_size_overdamped_point_vs_quadrature(lib):
    """gamma = 0.9, D = 0.2 at the full 2^20 trajectories: mean escape time vs the exact
    MFPT quadrature (3 SE plus 1 % for the Euler and discrete-monitoring bias at dt = 1e-3)."""
    d = workloads.overdamped_sweep()[11]
    with _engine(lib, chunk_steps=16384) as eng:
        rid, res = _run(eng, d, d["n_traj"], d["seed"])
    T = mfpt.overdamped_mfpt(0.9, 0.2)
    assert res.n_used == 2**20 and res.n_censored == 0
    assert stats.within_combined_se(res.mean, res.sem, T, 0.0, 3.0, allowance=0.01 * T)


def test_errors(lib):
    with _engine(lib) as eng:
        with pytest.raises(lib.FptError) as ei:
            eng.poll(999)
        assert ei.value.status == -4
        with pytest.raises(lib.FptError):
            eng.submit(lib_params(CONST_OVER, precision="fp64"), 10, 1)
        with pytest.raises(lib.FptError):
            eng.submit(lib_params(CONST_OVER), 0, 1)
        with pytest.raises(lib.FptError):
            eng.submit(lib_params(CONST_OVER, hist_bins=0), 10, 1)
        rid = eng.submit(lib_params(CONST_OVER, max_steps=2**40), 100000, 1)
        eng.step(2)
        eng.release(rid)          # cancel while running
        eng.step(2)
        with pytest.raises(lib.FptError):
            eng.poll(rid)
        c = eng.counters()
        assert c["resident_requests"] == 0


def test_fair_share_no_starvation(lib):
    """A large request of short trajectories submitted first must not starve a small request of
    the same model submitted after it: as lanes free up, the exact per-request cap hands them to
    the newcomer."""
    big = workloads.scaled(CONST_OVER, D=0.2)
    with _engine(lib, chunk_steps=4096) as eng:
        hog = eng.submit(lib_params(big), 2**26, 1)
        eng.step(1)
        short = eng.submit(lib_params(CONST_OVER), 20000, 2)
        for _ in range(80):
            eng.step(1)
            st, res = eng.poll(short)
            if st == 0:
                break
        assert st == 0, "short request starved behind a never-ending one"
        c = eng.counters()
        assert c["escapes"] >= res.n_escaped > 0
        assert 0 < c["useful_steps"] <= c["lane_step_slots"]
        eng.release(hog)


RAMP = workloads.scaled(workloads.ramp_sweep(n_traj=1, rates=(1e-3,))[0], hist_bins=200,
                        hist_lo=0.5, hist_hi=1.5)


def test_engine_matches_plain_fp32_ramp(lib, api):
    """Ramped bias (Alg. 3): the bias is formed from each trajectory's own step count, so the
    engine and the plain kernel agree per trajectory here too."""
    n, seed = 3000, 77
    with _engine(lib, chunk_steps=1024) as eng:
        rid, res = _run(eng, RAMP, n, seed, keep_per_traj=1)
        e_steps = eng.per_traj_steps(rid, n)
    p_steps = api.run_plain(RAMP, n, seed).cpu().numpy()
    assert (e_steps == p_steps).all()


@pytest.mark.parametrize("hog_model", ["underdamped", "overdamped"])
def test_never_ending_request_does_not_starve(lib, hog_model):
    """A request that never finishes (no noise: every trajectory stays trapped) takes every lane
    first; a short request submitted later still completes, because lanes above the fair share
    are suspended (same model) and whole warps vacate (other model)."""
    hog = workloads.scaled(CONST_UNDER if hog_model == "underdamped" else CONST_OVER, D=0.0,
                           max_steps=2**40)
    with _engine(lib, chunk_steps=4096) as eng:
        h = eng.submit(lib_params(hog), 2**22, 1)
        eng.step(2)
        short = eng.submit(lib_params(CONST_OVER), 20000, 2)
        for _ in range(200):
            eng.step(1)
            st, res = eng.poll(short)
            if st == 0:
                break
        assert st == 0, "short request starved behind a never-ending one"
        assert eng.counters()["preempted"] > 0
        eng.release(h)


@pytest.mark.parametrize("target", [CONST_UNDER, RAMP], ids=["constant", "ramp"])
def test_suspended_trajectories_resume_exactly(lib, api, target):
    """Trajectories suspended by preemption and resumed later (possibly by another lane) give
    exactly the escape steps of an undisturbed run."""
    n, seed = 2**20, 99           # more trajectories than lanes: the target fills the GPU
    blocker = workloads.scaled(CONST_UNDER, D=0.0, max_steps=2**40)
    with _engine(lib, chunk_steps=2048) as eng:
        rid = eng.submit(lib_params(target, keep_per_traj=1), n, seed)
        eng.step(3)
        b = eng.submit(lib_params(blocker), 2**22, 5)   # starved newcomer: target must yield
        res = eng.wait(rid, 600.0)
        steps = eng.per_traj_steps(rid, n)
        c = eng.counters()
        eng.release(b)
    assert c["preempted"] > 0
    ref = api.run_plain(target, n, seed).cpu().numpy()
    assert (steps == ref).all()


@pytest.mark.parametrize("target", [CONST_UNDER, RAMP], ids=["constant", "ramp"])
@pytest.mark.parametrize("service", [0, 1])
def test_checkpoint_restore_is_exact(lib, api, target, service):
    """A request checkpointed mid-run (lanes suspended, state serialised, engine destroyed) and
    restored into a differently shaped engine finishes with exactly the per-trajectory steps and
    sums of an uninterrupted run."""
    import time
    n, seed = 2**20, 123          # more trajectories than lanes: some still unclaimed
    with _engine(lib, chunk_steps=2048, service_thread=service) as eng:
        rid = eng.submit(lib_params(target, keep_per_traj=1), n, seed)
        if service:
            time.sleep(0.01)
        else:
            eng.step(5)
        blob = eng.checkpoint(rid)
        with pytest.raises(lib.FptError):
            eng.poll(rid)             # released after the checkpoint
    assert len(blob) > 0
    with _engine(lib, chunk_steps=8192, traj_per_thread=1) as eng:
        rid2 = eng.restore(blob)
        res = eng.wait(rid2, 600.0)
        steps = eng.per_traj_steps(rid2, n)
        sums = eng.exact_sums(rid2)
    ref = api.run_plain(target, n, seed).cpu().numpy()
    assert (steps == ref).all()
    assert res.n_used == n
    s = stats.summarize(oracle.params_from(target), ref)
    assert res.n_escaped == s.n_escaped
    assert math.isclose(res.mean, s.mean, rel_tol=1e-12)


def test_checkpoint_of_queued_request(lib, api):
    """A request checkpointed before admission restores as a fresh run."""
    with _engine(lib, chunk_steps=2048, max_requests=1) as eng:
        first = eng.submit(lib_params(CONST_OVER), 1000, 1)
        queued = eng.submit(lib_params(CONST_OVER, keep_per_traj=1), 3000, 9)
        blob = eng.checkpoint(queued)        # still waiting for the only slot
        rid = eng.restore(blob)
        eng.wait(first, 600.0)
        eng.wait(rid, 600.0)
        steps = eng.per_traj_steps(rid, 3000)
    assert (steps == api.run_plain(CONST_OVER, 3000, 9).cpu().numpy()).all()


def test_admission_by_memory_budget(lib, api):
    """An engine whose device-memory budget holds one such request at a time queues the others
    (admitted as memory frees), finishes all of them with their exact results, and rejects a
    request that could never fit."""
    d = workloads.scaled(CONST_OVER, max_steps=10**8)
    n = 2**20                                  # keep_per_traj: 8 MB of per-trajectory steps
    with _engine(lib, chunk_steps=16384, mem_budget_bytes=22 << 20) as eng:
        ids = [eng.submit(lib_params(d, keep_per_traj=1), n, 40 + i) for i in range(3)]
        eng.step(1)
        c = eng.counters()
        assert c["resident_requests"] == 1 and c["pending_requests"] == 2
        got = []
        for rid in ids:
            eng.wait(rid, 600.0)
            got.append(eng.per_traj_steps(rid, n))
            eng.release(rid)
        with pytest.raises(lib.FptError) as ei:
            eng.submit(lib_params(d, keep_per_traj=1), 2**23, 1)
        assert ei.value.status == -2          # FPT_ENOMEM
    for i, g in enumerate(got):
        assert (g == api.run_plain(d, n, 40 + i).cpu().numpy()).all()


def test_restore_rejects_foreign_or_truncated_blobs(lib):
    """fpt_restore checks the blob: a wrong magic, another format version or a truncated buffer
    is rejected with FPT_EINVAL and leaves the engine usable."""
    import struct
    with _engine(lib, chunk_steps=2048) as eng:
        rid = eng.submit(lib_params(CONST_OVER), 4000, 3)
        eng.step(1)
        blob = eng.checkpoint(rid)
        magic, version = struct.unpack_from("<QQ", blob, 0)
        for bad in (struct.pack("<QQ", magic ^ 1, version) + blob[16:],
                    struct.pack("<QQ", magic, version + 1) + blob[16:],
                    blob[: len(blob) // 2]):
            with pytest.raises(lib.FptError) as ei:
                eng.restore(bad)
            assert ei.value.status == -1
        res = eng.wait(eng.restore(blob), 600.0)
        assert res.n_used == 4000


@pytest.mark.parametrize("integrator", ["em", "heun"])
def test_noise_free_running_state_period(lib, api, integrator):
    """D = 0, gamma = 1.5 > 1 (no well): every trajectory runs down the washboard and crosses
    phi0 + 2 pi after the running period 2 pi / sqrt(gamma^2 - 1) = 5.6199, i.e. at step
    ceil(T / dt) = 5620 of a per-step test (the FP64 oracle gives exactly that for both
    integrators); the FP32 engine lands within 3 steps, identically for every trajectory and for
    the plain kernel."""
    d = workloads.base(model="overdamped", D=0.0, gamma0=1.5, dt=1e-3, phi0=0.0,
                       threshold=2 * math.pi, threshold_mode="from_start", max_steps=10**6,
                       integrator=integrator)
    n = 3000
    with _engine(lib, chunk_steps=2048) as eng:
        rid = eng.submit(lib_params(d, keep_per_traj=1), n, 1)
        eng.wait(rid, 600.0)
        k = eng.per_traj_steps(rid, n)
    assert (k == k[0]).all()
    assert (k == api.run_plain(d, n, 1).cpu().numpy()).all()
    want = math.ceil(mfpt.running_period(1.5) / 1e-3)
    assert abs(int(k[0]) - want) <= 3, (k[0], want)


@pytest.mark.parametrize("output", ["time", "bias"])
def test_per_trajectory_observables_and_censoring(lib, output):
    """fpt_per_traj: x = k dt (time) or gamma0 + (nu dt) k (bias, Alg. 3) in IEEE double for
    every escaped trajectory, equal to the oracle's definition; censored trajectories (a budget
    that only part of them meets) are -1 (time) or NaN (bias), and counted in n_censored."""
    if output == "bias":
        d = workloads.scaled(RAMP, max_steps=98000)          # bias 0.98: about half switch
    else:
        d = workloads.scaled(CONST_UNDER, max_steps=200000)
    n = 4000
    with _engine(lib, chunk_steps=4096) as eng:
        rid = eng.submit(lib_params(d, keep_per_traj=1), n, 23)
        res = eng.wait(rid, 600.0)
        k = eng.per_traj_steps(rid, n)
        x = eng.per_traj(rid, n)
    p = oracle.params_from(d)
    cens = k < 0
    assert 0 < cens.sum() < n and res.n_censored == cens.sum()
    want = np.array([stats.observable(p, int(v)) for v in k[~cens]])
    assert (x[~cens] == want).all()
    if output == "bias":
        assert np.isnan(x[cens]).all()
    else:
        assert (x[cens] == -1.0).all()


@pytest.mark.parametrize("max_steps", [1, 3, 5, 17, 33])
def test_tiny_step_budgets(lib, api, max_steps):
    """Budgets shorter than, equal to and just past one 16-step block: the engine runs whole
    blocks, so it integrates past the budget and must count only escapes at k <= max_steps.
    Per trajectory it equals the plain kernel; the escape count per step matches the FP64
    oracle's within binomial noise, and nothing beyond the budget is counted."""
    d = workloads.base(model="overdamped", D=0.5, gamma0=0.5, dt=0.01, threshold=0.3,
                       threshold_mode="from_start", max_steps=max_steps)
    n = 20000
    with _engine(lib, chunk_steps=1024) as eng:
        rid, res = _run(eng, d, n, 9, keep_per_traj=1)
        k = eng.per_traj_steps(rid, n)
    assert (k == api.run_plain(d, n, 9).cpu().numpy()).all()
    assert k.max() <= max_steps and res.n_escaped == (k >= 0).sum()
    assert res.steps_total == int(k[k >= 0].sum()) + max_steps * int((k < 0).sum())
    r = oracle.run(oracle.params_from(d), 9, 4000)
    f_gpu, f_ref = (k >= 0).mean(), (r >= 0).mean()
    se = math.sqrt(max(f_ref * (1 - f_ref), 1e-4) / 4000 + max(f_gpu * (1 - f_gpu), 1e-4) / n)
    assert abs(f_gpu - f_ref) < 4 * se, (f_gpu, f_ref)


@pytest.mark.parametrize("integrator", ["em", "heun"])
def test_hundred_windings_to_the_threshold(lib, api, integrator):
    """D = 0, gamma = 1.5, threshold 100 periods (200 pi) from the start: the wrapped phase must
    count 99 upper wraps and then find the threshold in its cell.  The FP64 oracle (unwrapped
    phase) crosses at step 561 986 for both integrators.  The FP32 phase adds increments of
    ~1.5e-3 to values of order pi, so each step rounds at ~1e-4 of its increment; measured over
    these 5.6e5 steps that accumulates to 14 steps (2.5e-5 of the time), asserted below 1e-4."""
    d = workloads.base(model="overdamped", D=0.0, gamma0=1.5, dt=1e-3, phi0=0.0,
                       threshold=200 * math.pi, threshold_mode="from_start", max_steps=10**7,
                       integrator=integrator)
    p = oracle.params_from(d)
    esc, k_ref, *_ = oracle.trajectory(p, 0, 0)
    assert esc
    with _engine(lib, chunk_steps=16384) as eng:
        rid, res = _run(eng, d, 64, 1, keep_per_traj=1)
        k = eng.per_traj_steps(rid, 64)
    assert (k == k[0]).all() and (k == api.run_plain(d, 64, 1).cpu().numpy()).all()
    assert abs(int(k[0]) - k_ref) <= 1e-4 * k_ref, (k[0], k_ref)
