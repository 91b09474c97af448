"""CPU tests of the C ABI: the library loads, exports every declared symbol,
and its host-side planning and correctly rounded tables equal the oracle's."""
import os
import random
import re

import pytest

import workloads as wl
from conftest import ROOT
from oracle import plan, poly, search

tmd = pytest.importorskip("paper_1211_3056_gb300")


def declared_functions(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"\b(tmd_\w+)\s*\(", src))


def test_exports_every_declared_symbol():
    """include/tmd.h is libtmd.so's boundary, include/tmd_probe.h
    libtmd_probe.so's; every header of include/ is one of the two."""
    import ctypes
    assert sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")) == \
        ["tmd.h", "tmd_probe.h"]
    for header, path, sigs in (("tmd.h", tmd._lib.LIB_PATH, tmd._lib.SIGNATURES),
                               ("tmd_probe.h", tmd._lib.PROBE_PATH, tmd._lib.PROBE_SIGNATURES)):
        lib = ctypes.CDLL(path)
        names = declared_functions(header)
        assert len(names) >= (12 if header == "tmd.h" else 1)
        for n in sorted(names):
            assert hasattr(lib, n), (header, n)
        assert set(sigs) <= names
    assert "tmd_pipe_rates" not in declared_functions("tmd.h")


def test_version_and_status_strings():
    assert "sm_103a" in tmd.tmd_version()
    assert tmd._lib.status_str(0) == "ok"


def oracle_table(job, blk):
    W = 64 * job.limbs
    N = 1 << job.log2_N
    mod = 1 << W
    c = poly.taylor_coeffs(job, blk)
    g0 = [poly.horner(c, i * N, W) for i in range(job.d + 1)]
    g1 = [(poly.horner(c, i * N + 1, W) - poly.horner(c, i * N, W)) % mod for i in range(job.d)]
    t0 = [r[0] % mod for r in search.forward_differences(g0)]
    t1 = [r[0] % mod for r in search.forward_differences(g1)]
    return c, t0 + t1


HOST_JOBS = [
    wl.toy_job(),
    wl.plain_job(),
    wl.Job(wl.FUNC_EXP2, 1, 24, 16, 8, 2, 12, 1, 0, 1 << 12),
    wl.Job(wl.FUNC_EXP, 1, 53, 40, 12, 4, 20, 3, 1 << 40, 1 << 30),
    wl.Job(wl.FUNC_EXP, 2, 40, 30, 10, 3, 20, 2, 0, 1 << 39),             # three cuts (8, 16, 32)
    wl.Job(wl.FUNC_LOG, 2, 53, 40, 14, 3, 24, 3, 3 << 49, 1 << 44),        # crosses e
    wl.Job(wl.FUNC_LOG, 3, 30, 20, 8, 2, 12, 2, 0, 1 << 29, wl.FLAG_BP_DIRECTED),
    wl.Job(wl.FUNC_EXP2, 0, 53, 42, 16, 1, 20, 1, 12345 << 20, 1 << 24),
    wl.Job(wl.FUNC_EXP, -5, 53, 40, 14, 2, 18, 2, 999 << 18, 1 << 22),
    # range-reduced binades: exp on [128, 256) across the cut at 260 ln 2,
    # 2^x across X = 200, exp on [4, 8) with three cuts, the top binades
    wl.Job(wl.FUNC_EXP, 8, 53, 32, 16, 3, 20, 3, 1837266934047447 - (1 << 33), 1 << 34),
    wl.Job(wl.FUNC_EXP2, 8, 53, 32, 14, 3, 20, 3, (72 << 45) - (1 << 31), 1 << 32),
    wl.Job(wl.FUNC_EXP, 3, 40, 24, 10, 3, 20, 2, 0, 1 << 38),
    wl.Job(wl.FUNC_EXP2, 9, 30, 16, 8, 2, 12, 2, 5 << 19, 1 << 21, wl.FLAG_BP_DIRECTED),
    wl.Job(wl.FUNC_EXP, 9, 53, 40, 14, 3, 20, 3, (1 << 52) - (1 << 30), 1 << 30),
    # argument shifts p - e_in of 64 and more (X = M 2^-69, 2^-76), block
    # starts with many trailing zero bits: not integer arguments
    wl.Job(wl.FUNC_EXP2, -16, 53, 20, 14, 3, 20, 3, 1 << 40, 1 << 26),
    wl.Job(wl.FUNC_EXP, -16, 60, 24, 14, 3, 20, 3, 5 << 50, 1 << 26),
] + wl.batched_jobs()[:6]


@pytest.mark.parametrize("job", HOST_JOBS, ids=lambda j: f"f{j.func}e{j.e_in}p{j.p}d{j.d}L{j.limbs}")
def test_plan_and_tables_match_oracle(job):
    info = tmd.tmd_plan(job)
    ob = plan.blocks(job)
    assert info["n_blocks"] == len(ob)
    assert info["n_subints"] == plan.n_subintervals(job)
    assert info["cuts"] == [s[0] for s in plan.segments(job)[1:]]
    rng = random.Random(job.start ^ job.count)
    picks = sorted(set([0, len(ob) - 1] + [rng.randrange(len(ob)) for _ in range(4)]))
    for b in picks:
        c, tab, bi = tmd.tmd_block_tables(job, b)
        oc, ot = oracle_table(job, ob[b])
        assert (bi["start"], bi["length"], bi["first_sub"], bi["e_out"]) == \
            (ob[b].start, ob[b].length, ob[b].first_sub, ob[b].e_out)
        assert c == oc
        assert tab == ot


@pytest.mark.parametrize("log2_N", [2, 16])
@pytest.mark.parametrize("limbs", [1, 2, 3])
@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_difference_words_every_degree_width_and_length(d, limbs, log2_N):
    """The table words, formed from closed forms in the coefficients, equal
    the forward differences of Horner values for every degree and word
    width, at the shortest and a long sub-interval (N^j shifts past W)."""
    job = wl.Job(wl.FUNC_EXP, 1, 53, 30, log2_N, d, max(log2_N, 18), limbs, 12345 << 18, 1 << 20)
    ob = plan.blocks(job)
    for b in sorted({0, len(ob) - 1}):
        c, tab, _ = tmd.tmd_block_tables(job, b)
        oc, ot = oracle_table(job, ob[b])
        assert c == oc
        assert tab == ot


def test_toy_every_block_table():
    job = wl.toy_job()
    for b, blk in enumerate(plan.blocks(job)):
        if b % 7:
            continue
        c, tab, _ = tmd.tmd_block_tables(job, b)
        assert (c, tab) == oracle_table(job, blk)


@pytest.mark.parametrize("field,value,status", [
    ("m", 1, tmd._lib.TMD_EINVAL), ("m", 64, tmd._lib.TMD_EINVAL),
    ("log2_N", 17, tmd._lib.TMD_EUNSUPPORTED), ("d", 5, tmd._lib.TMD_EUNSUPPORTED),
    ("limbs", 4, tmd._lib.TMD_EUNSUPPORTED), ("count", 0, tmd._lib.TMD_EINVAL),
    ("start", 1 << 52, tmd._lib.TMD_EINVAL), ("e_in", 10, tmd._lib.TMD_EUNSUPPORTED),
    ("e_in", 46, tmd._lib.TMD_EUNSUPPORTED),
    ("log2_T", 13, tmd._lib.TMD_EINVAL), ("func", 7, tmd._lib.TMD_EINVAL),
    ("flags", 16, tmd._lib.TMD_EINVAL), ("flags", 8, tmd._lib.TMD_EINVAL), ("eps1", 5, tmd._lib.TMD_EINVAL)])
def test_validation(field, value, status):
    job = wl.plain_job().replace(**{field: value})
    if field == "log2_T":
        job = job.replace(log2_N=14)
    with pytest.raises(tmd.TmdError) as e:
        tmd.tmd_plan(job)
    assert e.value.status == status


@pytest.mark.parametrize("job,ok", [
    (wl.Job(wl.FUNC_LOG, 16, 12, 4, 2, 2, 4, 1, 0, 1 << 8), False),      # p - e_in < 1
    (wl.Job(wl.FUNC_EXP, 8, 15, 4, 2, 2, 4, 1, 0, 1 << 8), False),       # reduced binade, q < 8
    (wl.Job(wl.FUNC_EXP, 1, 8, 4, 2, 2, 4, 1, 0, 1 << 6), True),         # q = 7 on [1, 2)
    (wl.Job(wl.FUNC_EXP2, 8, 16, 4, 2, 2, 4, 1, 0, 1 << 8), True),       # q = 8 on [128, 256)
])
def test_argument_shift_limits(job, ok):
    if ok:
        tmd.tmd_plan(job)
    else:
        with pytest.raises(tmd.TmdError) as e:
            tmd.tmd_plan(job)
        assert e.value.status == tmd._lib.TMD_EUNSUPPORTED


def test_log_binade_near_one_rejected():
    job = wl.Job(wl.FUNC_LOG, 1, 53, 40, 14, 3, 24, 3, 0, 1 << 30)
    with pytest.raises(tmd.TmdError):
        tmd.tmd_plan(job)


SOUND_JOBS = [
    wl.Job(wl.FUNC_EXP, 1, 53, 32, 15, 3, 24, 3, 0, 1 << 39, wl.FLAG_BP_DIRECTED),
    wl.plain_job(),
    wl.Job(wl.FUNC_EXP, 0, 24, 10, 8, 2, 12, 1, 3 << 20, 1 << 13),
    wl.Job(wl.FUNC_EXP2, 1, 22, 7, 7, 3, 11, 1, 12345, 1 << 11, wl.FLAG_BP_DIRECTED),
    wl.Job(wl.FUNC_LOG, 2, 20, 8, 6, 2, 10, 1, 100, 1 << 12),
    wl.Job(wl.FUNC_LOG, 3, 53, 40, 16, 2, 18, 3, 1 << 44, 1 << 30),
    wl.Job(wl.FUNC_EXP, 0, 20, 7, 6, 2, 10, 2, 0, 1 << 19),
    wl.Job(wl.FUNC_EXP, 8, 53, 32, 16, 3, 20, 3, 1837266934047447 - (1 << 33), 1 << 34),
    wl.Job(wl.FUNC_EXP2, 8, 53, 32, 14, 3, 20, 3, (72 << 45) - (1 << 31), 1 << 32),
]


@pytest.mark.parametrize("job", SOUND_JOBS, ids=lambda j: f"f{j.func}p{j.p}N{j.log2_N}")
def test_sound_eps_not_below_the_oracle_bounds(job):
    """tmd_sound_eps (double precision with margins) never returns less than
    the oracle's exact-rational smallest sound thresholds, and not much more."""
    from oracle import sound
    e1, e3 = tmd.tmd_sound_eps(job)
    o1, o3 = sound.min_eps(job)
    assert e1 >= o1 and e3 >= o3
    assert e1 <= o1 * 1.01 + 64 and e3 <= o3 * 1.01 + 64


@pytest.mark.parametrize("job", SOUND_JOBS, ids=lambda j: f"f{j.func}p{j.p}N{j.log2_N}")
def test_sound_piece_eps_not_below_the_oracle_bound(job):
    from oracle import sound
    sj = tmd.sound_job(job)
    e2 = tmd.tmd_sound_piece_eps(sj)
    o2 = sound.min_eps2(job, sj.eps3)
    assert o2 <= e2 <= o2 * 1.01 + 64
    assert sj.eps3 < e2 < sj.eps1


@pytest.mark.parametrize("job", SOUND_JOBS, ids=lambda j: f"f{j.func}e{j.e_in}p{j.p}N{j.log2_N}")
def test_sound_line_eps_not_below_the_oracle_bound(job):
    """The half-width of the phase-3 sub-pieces (and of any line length)
    against the oracle's exact-rational bound; lengths outside 1..N refused."""
    from oracle import sound
    sj = tmd.sound_job(job)
    N = 1 << job.log2_N
    n2 = (N + 31) // 32
    for length in sorted({1, (n2 + 31) // 32, n2, N}):
        e = tmd.tmd_sound_line_eps(sj, length)
        o = sound.min_eps_len(job, sj.eps3, length)
        assert o <= e <= o * 1.01 + 64
    assert tmd.tmd_sound_line_eps(sj, n2) == tmd.tmd_sound_piece_eps(sj)
    for bad in (0, N + 1):
        with pytest.raises(tmd.TmdError):
            tmd.tmd_sound_line_eps(sj, bad)


def test_sound_job_validation():
    job = tmd.sound_job(wl.toy_job())
    tmd.tmd_plan(job)                                   # accepted
    for bad in (job.replace(eps3=1), job.replace(eps1=job.eps3), job.replace(eps1=1 << 62),
                job.replace(flags=job.flags | wl.FLAG_ALL_HITS), wl.toy_job().replace(eps3=5)):
        with pytest.raises(tmd.TmdError) as e:
            tmd.tmd_plan(bad)
        assert e.value.status == tmd._lib.TMD_EINVAL


def random_jobs(n, seed):
    """Seeded valid jobs over every supported (function, binade) range,
    precision, degree, width and length: exp and 2^x from [2^-16, 2^-15) to
    [256, 512), log from [2, 4) to [2^15, 2^16)."""
    rng = random.Random(seed)
    out = []
    while len(out) < n:
        func = rng.choice([wl.FUNC_EXP, wl.FUNC_EXP2, wl.FUNC_LOG])
        e_in = rng.randint(2, 16) if func == wl.FUNC_LOG else rng.choice([-16, -3, 0, 1, 2, 3, 5, 8, 9])
        p = rng.choice([24, 30, 40, 53])
        if p - e_in < (8 if func != wl.FUNC_LOG and e_in > 2 else 1):
            continue
        log2_N = rng.randint(2, 14)
        log2_T = log2_N + rng.randint(0, 8)
        d = rng.randint(1, 4)
        limbs = rng.randint(1, 3)
        span = 1 << (p - 1)
        count = rng.randint(1, min(span, 1 << rng.randint(4, 34)))
        start = rng.randrange(0, span - count + 1)
        job = wl.Job(func, e_in, p, rng.randint(8, 40), log2_N, d, log2_T, limbs, start, count,
                     rng.choice([0, wl.FLAG_BP_DIRECTED]))
        try:
            tmd.tmd_plan(job)
        except tmd.TmdError as e:
            # more than 4 output binades in the slice is the one refusal expected
            assert e.status == tmd._lib.TMD_EUNSUPPORTED
            continue
        out.append(job)
    return out


@pytest.mark.parametrize("job", random_jobs(16, 20261204), ids=lambda j: f"f{j.func}e{j.e_in}p{j.p}d{j.d}L{j.limbs}")
def test_random_plans_and_tables_match_oracle(job):
    info = tmd.tmd_plan(job)
    ob = plan.blocks(job)
    assert info["n_blocks"] == len(ob)
    assert info["n_subints"] == plan.n_subintervals(job)
    assert info["cuts"] == [s[0] for s in plan.segments(job)[1:]]
    rng = random.Random(job.start ^ job.count ^ 77)
    for b in sorted({0, len(ob) - 1, rng.randrange(len(ob))})[:3]:
        c, tab, bi = tmd.tmd_block_tables(job, b)
        oc_, ot = oracle_table(job, ob[b])
        assert bi["e_out"] == ob[b].e_out
        assert c == oc_ and tab == ot


def random_sound_jobs(n, seed):
    """Seeded valid jobs whose sound thresholds fit (eps1 < 2^62)."""
    rng = random.Random(seed)
    out = []
    for job in random_jobs(4 * n, seed):
        if len(out) == n:
            break
        if job.func == wl.FUNC_EXP2 and job.e_in > 3:
            continue  # keeps the oracle's 2^x enclosures short
        try:
            tmd.tmd_sound_eps(job)
        except tmd.TmdError as e:
            assert e.status == tmd._lib.TMD_EINVAL  # thresholds past 2^62 are refused
            continue
        out.append(job.replace(m=rng.randint(8, 40)))
    return out


@pytest.mark.parametrize("job", random_sound_jobs(10, 4242), ids=lambda j: f"f{j.func}e{j.e_in}p{j.p}d{j.d}")
def test_random_sound_eps_not_below_the_oracle_bounds(job):
    from oracle import sound
    try:
        e1, e3 = tmd.tmd_sound_eps(job)
    except tmd.TmdError as e:
        assert e.status == tmd._lib.TMD_EINVAL
        return
    o1, o3 = sound.min_eps(job)
    assert o3 <= e3 <= o3 * 1.01 + 64
    assert o1 <= e1 <= o1 * 1.01 + 64


def test_fuzzed_job_records_never_crash():
    """Random field values, mostly out of range: tmd_plan answers OK,
    TMD_EINVAL or TMD_EUNSUPPORTED, never anything else."""
    rng = random.Random(99)
    seen = set()
    for _ in range(3000):
        job = wl.Job(rng.choice([-1, 0, 1, 2, 3, 7]), rng.randint(-40, 80), rng.randint(-5, 70), rng.randint(-3, 70),
                     rng.randint(0, 40), rng.randint(-2, 9), rng.randint(0, 70), rng.randint(0, 6),
                     rng.getrandbits(rng.choice([0, 8, 40, 63, 64])), rng.getrandbits(rng.choice([0, 1, 20, 52, 64])),
                     rng.choice([0, 1, 2, 4, 8, 16, 3, 12]))
        try:
            tmd.tmd_plan(job)
            seen.add(0)
        except tmd.TmdError as e:
            assert e.status in (tmd._lib.TMD_EINVAL, tmd._lib.TMD_EUNSUPPORTED), (job, e.status)
            seen.add(e.status)
        except (OverflowError, ValueError, TypeError):
            seen.add(-1)  # not representable in the C record: refused by the binding
    assert tmd._lib.TMD_EINVAL in seen and tmd._lib.TMD_EUNSUPPORTED in seen
