"""The continuous-batching server: results alone vs in a mix, agreement with a
direct engine run, and admission by device-memory footprint."""

import numpy as np
import pytest

import oracle as orc
from paper_2408_13782_gb300 import Engine, FpmError
from paper_2408_13782_gb300 import serve as sv
from synth import recipes as S
from tests.gpu_common import record
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu


def _job(N, grid, seed, max_epochs=6, rel_tol=0.0, c=None):
    """A serving request (the 64-px recipe scaled to N) with a stack simulated by the engine."""
    c = c if c is not None else S.serving_job_config(N, grid, seed)
    nominal, truth = S.led_grid(c.grid, c.pitch, c.jitter, c.seed)
    eng = Engine(c.m, c.s, truth, c.R, c.lambda_um, c.dk_per_um, c.edge)
    eng.set_object_field(S.make_object(c.N, c.seed))
    stack = eng.forward(np.arange(c.n_leds))
    eng.close()
    desc = sv.job_desc(c.m, c.s, nominal, c.R, c.lambda_um, c.dk_per_um, c.edge, batch=c.B,
                       max_epochs=max_epochs, rel_tol=rel_tol, seed=c.seed, lr=dict(object=0.5))
    return c, desc, stack


def _serve(jobs, budget=8 << 30, max_active=16, grouping="config"):
    srv = sv.Server(budget, max_active, grouping=grouping)
    ids, st, wall = sv.run_arrivals(srv, [(d, s, t) for (c, d, s), t in jobs])
    res = [srv.result(i, c.N, c.n_leds) for i, ((c, d, s), t) in zip(ids, jobs)]
    srv.close()
    return st, res


def test_result_alone_equals_result_in_a_mix():
    a = _job(512, 11, 5)
    others = [_job(256, 7, 6), _job(1024, 7, 7), _job(256, 15, 8)]
    st_alone, res_alone = _serve([(a, 0.0)])
    st_mix, res_mix = _serve([(others[0], 0.0), (a, 0.0), (others[1], 0.0), (others[2], 0.002)])
    assert st_alone[0]["state"] == sv.JOB_DONE and st_mix[1]["state"] == sv.JOB_DONE
    assert st_alone[0]["epochs"] == st_mix[1]["epochs"] == 6
    assert np.array_equal(res_alone[0]["object"], res_mix[1]["object"])
    assert abs(st_alone[0]["loss"] - st_mix[1]["loss"]) <= 1e-12 * abs(st_alone[0]["loss"])
    # the jobs of the mix overlapped on the device
    t_admit = [s["t_admit"] for s in st_mix]
    t_done = [s["t_done"] for s in st_mix]
    assert max(t_admit) < min(t_done)


def test_served_job_equals_a_direct_run():
    c, desc, stack = _job(256, 11, 9, max_epochs=4)
    st, res = _serve([((c, desc, stack), 0.0)])
    nominal = S.led_grid(c.grid, c.pitch, c.jitter, c.seed)[0]
    eng = Engine(c.m, c.s, nominal, c.R, c.lambda_um, c.dk_per_um, c.edge)
    eng.set_hparams(lr=dict(object=0.5))
    eng.load(stack, init=True)
    for e in range(4):   # the server's epoch: full batches, then the short one
        perm = S.epoch_permutation(c.n_leds, c.seed, e)
        nfull = c.n_leds // c.B
        eng.run(perm[:nfull * c.B].reshape(nfull, c.B))
        if c.n_leds % c.B:
            eng.step(perm[nfull * c.B:])
    assert np.array_equal(eng.get()["object"], res[0]["object"])


def test_served_jobs_with_other_optimisers_equal_direct_runs():
    """Rounds whose jobs share Adam use the serving update kernel with the rule
    fixed at compile time; a round that holds an AdamW job and a NAdam job
    branches per job. Each served result equals a direct engine run bit for bit."""
    specs = [("adamw", 0.01, 50), ("nadam", 0.0, 51)]
    jobs = []
    for opt, wd, seed in specs:
        c = S.serving_job_config(256, 7, seed)
        nominal, truth = S.led_grid(c.grid, c.pitch, c.jitter, c.seed)
        eng = Engine(c.m, c.s, truth, c.R, c.lambda_um, c.dk_per_um, c.edge)
        eng.set_object_field(S.make_object(c.N, c.seed))
        stack = eng.forward(np.arange(c.n_leds))
        eng.close()
        desc = sv.job_desc(c.m, c.s, nominal, c.R, c.lambda_um, c.dk_per_um, c.edge, batch=c.B, max_epochs=3,
                           rel_tol=0.0, seed=c.seed, lr=dict(object=0.5), optimizer=opt, weight_decay=wd)
        jobs.append(((c, desc, stack), nominal, opt, wd))
    st, res = _serve([(j[0], 0.0) for j in jobs])
    for ((c, desc, stack), nominal, opt, wd), r, x in zip(jobs, res, st):
        assert x["state"] == sv.JOB_DONE and x["epochs"] == 3
        eng = Engine(c.m, c.s, nominal, c.R, c.lambda_um, c.dk_per_um, c.edge)
        eng.set_hparams(lr=dict(object=0.5), optimizer=opt, weight_decay=wd)
        eng.load(stack, init=True)
        for e in range(3):
            perm = S.epoch_permutation(c.n_leds, c.seed, e)
            nfull = c.n_leds // c.B
            eng.run(perm[:nfull * c.B].reshape(nfull, c.B))
            if c.n_leds % c.B:
                eng.step(perm[nfull * c.B:])
        assert np.array_equal(eng.get()["object"], r["object"]), opt
        eng.close()


def test_served_job_equals_the_oracle():
    """A served job against the FP64 oracle's reconstruction on the same schedule:
    each epoch a fresh permutation (Eq. 13-14), its full batches, then the short one."""
    c, desc, stack = _job(256, 7, 13, max_epochs=2)
    st, res = _serve([((c, desc, stack), 0.0)])
    assert st[0]["state"] == sv.JOB_DONE and st[0]["epochs"] == 2
    nominal = S.led_grid(c.grid, c.pitch, c.jitter, c.seed)[0]
    g = orc.Geometry(c.N, c.m, nominal, c.R, c.edge, c.lambda_um, c.dk_per_um)
    rec = orc.Reconstruction(g, stack, orc.Hparams(lr=dict(object=0.5), learn=("object",)))
    losses = []
    for e in range(2):
        perm = S.epoch_permutation(c.n_leds, c.seed, e)
        batches = [perm[k:k + c.B] for k in range(0, c.n_leds, c.B)]
        losses.append(sum(rec.run(batches)))
    err = rel_l2(res[0]["object"], rec.O)
    record("serving.m64.object", err)
    assert err <= 1e-3, err
    assert abs(st[0]["loss"] - losses[-1]) <= 1e-5 * losses[-1]


def test_rgb_channels_co_scheduled_equal_their_solo_runs():
    """Section 3.3's colour workflow: the three wavelengths of one field of view as
    three jobs with the same stack shape submitted together; they overlap on the
    device, and each channel's result equals the channel served alone, bit for bit."""
    chans = [_job(512, 11, 0, max_epochs=4, c=c) for c in S.rgb_job_configs(512, 11, 17)]
    st_mix, res_mix = _serve([(j, 0.0) for j in chans])
    assert all(x["state"] == sv.JOB_DONE and x["epochs"] == 4 for x in st_mix)
    assert max(x["t_admit"] for x in st_mix) < min(x["t_done"] for x in st_mix)   # co-resident
    for j, r in zip(chans, res_mix):
        st1, res1 = _serve([(j, 0.0)])
        assert np.array_equal(res1[0]["object"], r["object"])
    # the channels differ (different pupils and LED geometries), as they should
    assert not np.array_equal(res_mix[0]["object"], res_mix[2]["object"])


def test_admission_waits_for_memory():
    big1, big2 = _job(1024, 11, 10, max_epochs=3), _job(1024, 11, 11, max_epochs=3)
    small = _job(256, 7, 12, max_epochs=3)
    fp_big, fp_small = sv.footprint(big1[1]), sv.footprint(small[1])
    budget = fp_big + fp_small + (fp_big // 2)   # room for one big and one small job
    st, res = _serve([(big1, 0.0), (big2, 0.0), (small, 0.0)], budget=budget)
    assert all(s["state"] == sv.JOB_DONE for s in st)
    assert st[1]["t_admit"] >= st[0]["t_done"]       # the second big job waited for memory
    assert st[2]["t_admit"] < st[0]["t_done"]        # the small one did not
    with pytest.raises(Exception):                    # a job larger than the whole budget is refused
        srv = sv.Server(fp_small, 4)
        srv.submit(big1[1], big1[2])


def test_same_shape_jobs_share_rounds_and_match_alone():
    """Jobs of the same shape run in one round (one launch per step for all of
    them); each result equals the job served alone, bit for bit."""
    jobs = [_job(256, 7, 20 + k) for k in range(3)]
    srv = sv.Server(8 << 30, 16)
    ids, st, wall = sv.run_arrivals(srv, [(d, s, 0.0) for c, d, s in jobs])
    stats = srv.stats()
    res = [srv.result(i, c.N, c.n_leds) for i, (c, d, s) in zip(ids, jobs)]
    srv.close()
    assert all(x["state"] == sv.JOB_DONE for x in st)
    assert stats["max_jobs_per_round"] == 3
    assert stats["round_epochs"] == sum(x["epochs"] for x in st)
    for job, r in zip(jobs, res):
        st1, res1 = _serve([(job, 0.0)])
        assert np.array_equal(res1[0]["object"], r["object"])
        assert np.array_equal(res1[0]["gamma"], r["gamma"])


def test_mixed_sizes_share_one_launch_and_match_alone():
    """Jobs of low-res size 64, 128 and 256 with the same number of steps per
    epoch run in one round: one per-LED launch per step for all of them, their
    LEDs sharing clusters of 16 CTAs (4, 8 or 16 CTAs per LED). Each result
    equals the job served alone, bit for bit; the m = 64 job (the same CTA
    layout as the single-job kernel) equals a direct engine run bit for bit, and
    the m = 128 job (128-thread CTAs instead of 256) within FP32 rounding."""
    jobs = [_job(256, 7, 40, max_epochs=3), _job(512, 7, 41, max_epochs=3), _job(1024, 7, 42, max_epochs=3)]
    srv = sv.Server(8 << 30, 16, grouping="mixed")
    ids, st, wall = sv.run_arrivals(srv, [(d, s, 0.0) for c, d, s in jobs])
    stats = srv.stats()
    res = [srv.result(i, c.N, c.n_leds) for i, (c, d, s) in zip(ids, jobs)]
    srv.close()
    assert all(x["state"] == sv.JOB_DONE and x["epochs"] == 3 for x in st)
    assert stats["max_jobs_per_round"] == 3
    assert stats["round_epochs"] == 9
    for job, r in zip(jobs, res):
        st1, res1 = _serve([(job, 0.0)], grouping="mixed")
        assert np.array_equal(res1[0]["object"], r["object"])
        assert np.array_equal(res1[0]["gamma"], r["gamma"])
    for (c, desc, stack), r, exact in zip(jobs[:2], res[:2], (True, False)):
        nominal = S.led_grid(c.grid, c.pitch, c.jitter, c.seed)[0]
        eng = Engine(c.m, c.s, nominal, c.R, c.lambda_um, c.dk_per_um, c.edge)
        eng.set_hparams(lr=dict(object=0.5))
        eng.load(stack, init=True)
        for e in range(3):
            perm = S.epoch_permutation(c.n_leds, c.seed, e)
            nfull = c.n_leds // c.B
            eng.run(perm[:nfull * c.B].reshape(nfull, c.B))
            if c.n_leds % c.B:
                eng.step(perm[nfull * c.B:])
        O = eng.get()["object"]
        eng.close()
        if exact:
            assert np.array_equal(O, r["object"])
        else:
            assert rel_l2(r["object"], O) <= 1e-4


def test_grouping_policies_give_the_same_results():
    """The three grouping policies put the same jobs in different rounds (by
    kernel configuration, by size, sizes mixed); each job's result is the same
    under the size and mixed policies bit for bit (the same mixed-size launch
    body), and within rounding under the configuration policy; the policy
    cannot change while jobs are resident."""
    jobs = [_job(256, 7, 45, max_epochs=2), _job(256, 7, 46, max_epochs=2), _job(1024, 7, 47, max_epochs=2)]
    out = {}
    for pol in ("config", "size", "mixed"):
        st, res = _serve([(j, 0.0) for j in jobs], grouping=pol)
        assert all(x["state"] == sv.JOB_DONE for x in st)
        out[pol] = res
    for k in range(3):
        assert np.array_equal(out["size"][k]["object"], out["mixed"][k]["object"])
        assert rel_l2(out["config"][k]["object"], out["size"][k]["object"]) <= 1e-4
    assert np.array_equal(out["config"][0]["object"], out["size"][0]["object"])   # m = 64: the same layout
    srv = sv.Server(8 << 30, 4)
    c, d, s = jobs[0]
    srv.submit(d, s)
    srv.tick()
    with pytest.raises(FpmError):
        srv.set_grouping("mixed")
    srv.close()


def test_served_job_with_a_learned_pupil_field():
    """A job that learns the free-form pupil field beside the object runs the
    field's instantiation of the serving launches (same-configuration and
    mixed-size); both equal a direct engine run of its schedule bit for bit
    (m = 64: the same CTA layout in all three)."""
    c = S.serving_job_config(256, 7, 48)
    nominal, truth = S.led_grid(c.grid, c.pitch, c.jitter, c.seed)
    eng = Engine(c.m, c.s, truth, c.R, c.lambda_um, c.dk_per_um, c.edge)
    eng.set_object_field(S.make_object(c.N, c.seed))
    stack = eng.forward(np.arange(c.n_leds))
    eng.close()
    lr = dict(object=0.5, pupil=0.02)
    desc = sv.job_desc(c.m, c.s, nominal, c.R, c.lambda_um, c.dk_per_um, c.edge, batch=c.B, max_epochs=3,
                       rel_tol=0.0, seed=c.seed, lr=lr, learn=("object", "pupil"))
    res = {}
    for pol in ("config", "mixed"):
        st, r = _serve([((c, desc, stack), 0.0)], grouping=pol)
        assert st[0]["state"] == sv.JOB_DONE and st[0]["epochs"] == 3
        res[pol] = r[0]["object"]
    eng = Engine(c.m, c.s, nominal, c.R, c.lambda_um, c.dk_per_um, c.edge)
    eng.set_hparams(lr=lr, learn=("object", "pupil"))
    eng.load(stack, init=True)
    for e in range(3):
        perm = S.epoch_permutation(c.n_leds, c.seed, e)
        nfull = c.n_leds // c.B
        eng.run(perm[:nfull * c.B].reshape(nfull, c.B))
        if c.n_leds % c.B:
            eng.step(perm[nfull * c.B:])
    O = eng.get()["object"]
    P, on = eng.get_pupil()
    eng.close()
    assert on and np.max(np.abs(P - 1)) > 1e-4          # the field moved
    assert np.array_equal(res["config"], O)
    assert np.array_equal(res["mixed"], O)


def test_mixed_size_job_equals_the_oracle():
    """An m = 128 job served in a mixed-size round (beside an m = 256 job)
    against the FP64 oracle's reconstruction on the same schedule. The object
    is held to the spec trajectory bar (1e-3); the reported loss is the
    second epoch's, summed over batches taken after FP32 updates whose rounding
    Adam amplifies, so it is held to 1e-4."""
    a, b = _job(512, 7, 43, max_epochs=2), _job(1024, 7, 44, max_epochs=2)
    st, res = _serve([(a, 0.0), (b, 0.0)], grouping="mixed")
    c, desc, stack = a
    assert st[0]["state"] == sv.JOB_DONE and st[0]["epochs"] == 2
    nominal = S.led_grid(c.grid, c.pitch, c.jitter, c.seed)[0]
    g = orc.Geometry(c.N, c.m, nominal, c.R, c.edge, c.lambda_um, c.dk_per_um)
    rec = orc.Reconstruction(g, stack, orc.Hparams(lr=dict(object=0.5), learn=("object",)))
    losses = []
    for e in range(2):
        perm = S.epoch_permutation(c.n_leds, c.seed, e)
        losses.append(sum(rec.run([perm[k:k + c.B] for k in range(0, c.n_leds, c.B)])))
    err = rel_l2(res[0]["object"], rec.O)
    record("serving.mixed.m128.object", err)
    record("serving.mixed.m128.loss", abs(st[0]["loss"] - losses[-1]) / losses[-1])
    # the same schedule run directly (the single-job kernel, 256-thread CTAs): the
    # reference for how far FP32 rounding alone carries this trajectory
    eng = Engine(c.m, c.s, nominal, c.R, c.lambda_um, c.dk_per_um, c.edge)
    eng.set_hparams(lr=dict(object=0.5))
    eng.load(stack, init=True)
    for e in range(2):
        perm = S.epoch_permutation(c.n_leds, c.seed, e)
        nfull = c.n_leds // c.B
        eng.run(perm[:nfull * c.B].reshape(nfull, c.B))
        if c.n_leds % c.B:
            eng.step(perm[nfull * c.B:])
    record("serving.direct.m128.object", rel_l2(eng.get()["object"], rec.O))
    eng.close()
    assert err <= 1e-3, err
    assert abs(st[0]["loss"] - losses[-1]) <= 1e-4 * losses[-1]


def test_tensor_core_form_job_runs_beside_rounds():
    """A job in a tensor-core DFT form runs its own epochs (outside the rounds)
    next to same-shape FFT jobs, and equals a direct run of its form."""
    c, desc_fft, stack = _job(256, 7, 30, max_epochs=3)
    nominal = S.led_grid(c.grid, c.pitch, c.jitter, c.seed)[0]
    desc_tc = sv.job_desc(c.m, c.s, nominal, c.R, c.lambda_um, c.dk_per_um, c.edge, batch=c.B, max_epochs=3,
                          rel_tol=0.0, seed=c.seed, lr=dict(object=0.5), precision="bf16x3")
    other = _job(256, 7, 31, max_epochs=3)
    srv = sv.Server(8 << 30, 16)
    ids, st, wall = sv.run_arrivals(srv, [(desc_tc, stack, 0.0), (desc_fft, stack, 0.0), (other[1], other[2], 0.0)])
    res = srv.result(ids[0], c.N, c.n_leds)
    stats = srv.stats()
    srv.close()
    assert all(x["state"] == sv.JOB_DONE for x in st)
    assert stats["max_jobs_per_round"] == 2          # the two FFT jobs; the tensor-core job ran on its own
    eng = Engine(c.m, c.s, nominal, c.R, c.lambda_um, c.dk_per_um, c.edge)
    eng.set_hparams(lr=dict(object=0.5), precision="bf16x3")
    eng.load(stack, init=True)
    for e in range(3):
        perm = S.epoch_permutation(c.n_leds, c.seed, e)
        nfull = c.n_leds // c.B
        eng.run(perm[:nfull * c.B].reshape(nfull, c.B))
        if c.n_leds % c.B:
            eng.step(perm[nfull * c.B:])
    assert np.array_equal(eng.get()["object"], res["object"])
