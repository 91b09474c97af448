// C-ABI entry points (include/tmd.h): context, plan residency, uploads,
// launches and read-back.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cstdlib>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <string>
#include <mutex>
#include <thread>
#include <vector>

#include "coeffs.cuh"
#include "dev.hpp"
#include "host.hpp"
#include "planrec.cuh"

namespace tmd {
cudaError_t launch_tasks(bool fused, uint32_t L, uint32_t D, bool G, const LaunchArgs& a, cudaStream_t s);
cudaError_t launch_persistent(uint32_t L, uint32_t D, bool G, const LaunchArgs& a, int ctas, cudaStream_t s);
cudaError_t persistent_occupancy(uint32_t L, uint32_t D, bool G, int* blocks_per_sm);
cudaError_t upload_coeff_consts(const CoeffConsts& C);
cudaError_t launch_block_tables(const DevJob* jobs, const DevBlock* blocks, uint64_t n_blocks, uint64_t* tables,
                                uint32_t* status, uint32_t* err, const uint64_t* ctab, uint32_t func_mask,
                                cudaStream_t s);
cudaError_t launch_coeff_tables(uint64_t* ctab, uint32_t* err, cudaStream_t s);
cudaError_t launch_plan(const DevJob* jobs, uint32_t n_jobs, DevBlock* blocks, uint64_t n_blocks,
                        const uint32_t* class_jobs, const uint64_t* class_task0, uint32_t n_entries,
                        DevTask* tasks, uint64_t n_tasks, uint32_t* plan_err, uint64_t* misc, uint32_t n_misc,
                        uint64_t* count, cudaStream_t s);
cudaError_t launch_zero_counters(uint64_t* misc, uint32_t n_misc, uint64_t* count, cudaStream_t s);
cudaError_t launch_readback(const uint64_t* count, const uint32_t* words, uint64_t* host, cudaStream_t s);
cudaError_t launch_plan_inline(const InlinePlan& src, uint32_t n_words, uint64_t* arena, uint32_t n_jobs,
                               uint64_t o_cjobs, uint64_t o_ctask, uint32_t n_entries, uint64_t o_blocks,
                               uint64_t n_blocks, uint64_t o_tasks, uint64_t n_tasks, uint32_t* plan_err,
                               uint64_t* misc, uint32_t n_misc, uint64_t* count, cudaStream_t s);
}  // namespace tmd

namespace tmd {
cudaError_t launch_search_lines(bool raw, const LineArgs& a, cudaStream_t s);
cudaError_t launch_lower_bounds(int mode, const uint64_t* B, const uint64_t* A, const uint32_t* len, uint64_t n,
                                uint64_t* lb, uint32_t* hs, uint32_t* err, cudaStream_t s);
}  // namespace tmd

using namespace tmd;

namespace {

struct ClassRange {
    uint32_t L, D;
    bool G;                 // general kernel variant (Lefevre filter or sound mode)
    uint64_t first, count;  // task range
};

// A plan: per-job records with their segment tables, the class grouping of
// the tasks, and (host mode only) the materialised blocks, tasks and tables.
struct Plan {
    std::vector<tmd_job> key;
    std::vector<DevJob> jobs;
    std::vector<uint32_t> class_jobs;   // job indices grouped by (limbs, degree) class
    std::vector<uint64_t> class_task0;  // global first task of each class_jobs entry
    std::vector<DevBlock> blocks;       // host mode
    std::vector<uint64_t> tables;       // host mode
    std::vector<DevTask> tasks;         // host mode
    std::vector<ClassRange> classes;
    uint64_t total_lines = 0;
    uint64_t total_args = 0;
    uint64_t table_words = 0;
    uint64_t n_blocks = 0;
    uint64_t n_tasks = 0;
    bool host_tables = true;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Kernel variant of a job: the general one for Lefevre's filter, the sound
// mode, and literal thresholds dense enough that a line fails the filter
// often (2^(65-m) N >= 2^57, about one line in 2^7 holding a value below the
// threshold): the general variant resolves a task's failing lines 32 at a
// time instead of round by round.  The plain variant keeps the sparse
// thresholds, where a line fails one time in 10^5 or less.
bool general_variant(uint32_t flags, int m, uint32_t log2_N) {
    return (flags & (TMD_LEFEVRE | TMD_SOUND)) != 0 || 65 - m + (int)log2_N >= 57;
}

}  // namespace

struct tmd_ctx {
    int device = 0;
    int sms = 0;
    // device arena holding the resident plan
    char* d_arena = nullptr;
    size_t arena_cap = 0;
    size_t off_jobs = 0, off_blocks = 0, off_tables = 0, off_tasks = 0;
    // counters: stats[5] u64, err u32, queue head u32
    uint64_t* d_misc = nullptr;
    // tables of the table-driven exp and 2^x enclosures (CT_WORDS words)
    uint64_t* d_ctab = nullptr;
    // pinned staging for uploads
    char* h_stage = nullptr;
    size_t stage_cap = 0;
    cudaEvent_t stage_done = nullptr;
    bool stage_pending = false;
    // mapped pinned landing words of the result read-back (count, error
    // words) and their device address
    uint64_t* h_small = nullptr;
    uint64_t* d_small = nullptr;
    Plan plan;
    bool resident = false;
    uint64_t upload_bytes = 0;
    const uint64_t* last_count = nullptr;
    // tilings chosen by tmd_autotune, by batch signature (tiling_key)
    std::mutex tune_mu;
    std::map<std::string, tmd_tiling> tuned;
};

namespace {

uint64_t* stats_ptr(tmd_ctx* c) { return c->d_misc; }
uint32_t* err_ptr(tmd_ctx* c) { return (uint32_t*)(c->d_misc + ST_COUNT); }
uint32_t* queue_ptr(tmd_ctx* c) { return (uint32_t*)(c->d_misc + ST_COUNT) + 1; }
uint32_t* plan_err_ptr(tmd_ctx* c) { return (uint32_t*)(c->d_misc + ST_COUNT) + 2; }

#define CK(x)                                  \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) return TMD_ECUDA; \
    } while (0)

unsigned host_threads() {
    const char* env = getenv("TMD_HOST_THREADS");
    if (env && atoi(env) > 0) return (unsigned)atoi(env);
    unsigned n = std::thread::hardware_concurrency();
    return n ? n : 1;
}

// A pool of host threads that stay parked between parallel runs (creating
// threads for every plan costs ~10-20 us each).  run(n, fn) executes fn on
// n threads, the caller being one of them; one run at a time (a second
// caller meanwhile gets fresh threads).  The pool is never destroyed: its
// parked threads end with the process.
class HostPool {
   public:
    static HostPool& get() {
        static HostPool* p = new HostPool();
        return *p;
    }
    bool try_run(unsigned n, const std::function<void()>& fn) {
        std::unique_lock<std::mutex> run_lk(run_mu_, std::try_to_lock);
        if (!run_lk.owns_lock()) return false;
        const unsigned helpers = n - 1;
        {
            std::lock_guard<std::mutex> lk(mu_);
            while (workers_.size() < helpers) workers_.emplace_back([this] { loop(); });
            fn_ = &fn;
            want_ = helpers;
            taken_ = 0;
            done_ = 0;
            gen_++;
        }
        cv_work_.notify_all();
        fn();
        std::unique_lock<std::mutex> lk(mu_);
        cv_done_.wait(lk, [&] { return done_ == want_; });
        fn_ = nullptr;
        return true;
    }

   private:
    void loop() {
        uint64_t seen = 0;
        std::unique_lock<std::mutex> lk(mu_);
        for (;;) {
            cv_work_.wait(lk, [&] { return gen_ != seen && taken_ < want_; });
            seen = gen_;
            taken_++;
            const std::function<void()>* f = fn_;
            lk.unlock();
            (*f)();
            lk.lock();
            if (++done_ == want_) cv_done_.notify_all();
        }
    }
    std::mutex run_mu_, mu_;
    std::condition_variable cv_work_, cv_done_;
    std::vector<std::thread> workers_;
    const std::function<void()>* fn_ = nullptr;
    uint64_t gen_ = 0;
    unsigned want_ = 0, taken_ = 0, done_ = 0;
};

// fn() on n threads (the calling thread alone when n <= 1)
template <class F>
void run_threads(unsigned n, F&& fn) {
    if (n <= 1) {
        fn();
        return;
    }
    const std::function<void()> f = fn;
    if (HostPool::get().try_run(n, f)) return;
    std::vector<std::thread> th;
    for (unsigned i = 0; i < n; i++) th.emplace_back(fn);
    for (auto& t : th) t.join();
}

// Lines per packet of a job.  Sound jobs whose first filter fails on most
// lines (half-width eps1 over N arguments covering a quarter of the unit or
// more: the binades where the degree-1 truncation dwarfs eps) take one line
// per packet whatever the tiling: each line then carries phases 2 and 3,
// and 32-line tasks keep the warps of the grid evenly loaded.
uint32_t choose_nu(const tmd_job& job, uint64_t n_sub_block, uint32_t nu_max) {
    const char* env = getenv("TMD_NU");
    uint32_t nu = 8;  // at most the kernels' shared-memory stage (8 lines per lane)
    if (nu_max) nu = nu_max;
    else if (env && atoi(env) > 0) nu = (uint32_t)atoi(env);
    if ((job.flags & TMD_SOUND) && (job.eps1 >> (61 - job.log2_N)) != 0) nu = 1;
    if (nu > 8) nu = 8;
    if (nu > n_sub_block) nu = (uint32_t)n_sub_block;
    if (nu < 1) nu = 1;
    return nu;
}

// Plan every job: output-binade segments and, per segment, its blocks,
// sub-intervals and packets, as counts and offsets in the job record (the
// device planning kernels expand them).  With host_tables the blocks, tasks
// and correctly rounded tables are also materialised on the host (threads
// over blocks).
tmd_status build_plan(const tmd_job* jobs, uint32_t njobs, Plan& P, bool host_tables = true, uint32_t nu_max = 0) {
    // reuse the vectors' storage of a previous plan (no new pages per call)
    P.key.clear();
    P.jobs.clear();
    P.class_jobs.clear();
    P.class_task0.clear();
    P.blocks.clear();
    P.tables.clear();
    P.tasks.clear();
    P.classes.clear();
    P.total_lines = P.total_args = P.table_words = P.n_blocks = P.n_tasks = 0;
    if (njobs == 0 || !jobs) return TMD_EINVAL;
    P.host_tables = host_tables;
    P.key.assign(jobs, jobs + njobs);
    // validation and output-binade cuts of every job (independent per job:
    // spread over host threads for large batches)
    std::vector<std::array<Segment, MAX_SEGMENTS>> seg_of(njobs);
    std::vector<uint8_t> nseg_of(njobs, 0);
    std::vector<tmd_status> st_of(njobs, TMD_OK);
    auto seg_work = [&](uint32_t a, uint32_t b) {
        std::vector<Segment> sg;
        for (uint32_t j = a; j < b; j++) {
            tmd_status st = validate_job(jobs[j]);
            if (st == TMD_OK) st = plan_segments(jobs[j], sg);
            if (st == TMD_OK && sg.size() > MAX_SEGMENTS) st = TMD_EUNSUPPORTED;
            st_of[j] = st;
            if (st != TMD_OK) continue;
            nseg_of[j] = (uint8_t)sg.size();
            for (size_t k = 0; k < sg.size(); k++) seg_of[j][k] = sg[k];
        }
    };
    const unsigned nth = njobs >= 128 ? std::min<unsigned>({host_threads(), 32u, njobs / 32}) : 1;
    std::atomic<uint32_t> next_chunk(0);
    run_threads(nth, [&]() {
        for (;;) {
            const uint32_t a = next_chunk.fetch_add(32);
            if (a >= njobs) break;
            seg_work(a, std::min<uint32_t>(njobs, a + 32));
        }
    });
    std::vector<Segment> segs;
    uint64_t line = 0, packet = 0, toff = 0, nblk_total = 0;
    for (uint32_t j = 0; j < njobs; j++) {
        const tmd_job& jb = jobs[j];
        if (st_of[j] != TMD_OK) return st_of[j];
        segs.assign(seg_of[j].begin(), seg_of[j].begin() + nseg_of[j]);
        DevJob dj;
        memset(&dj, 0, sizeof dj);
        const bool sound = (jb.flags & TMD_SOUND) != 0;
        dj.shift = sound ? jb.eps1 : 1ull << (64 - jb.m);
        dj.Tm = 2 * dj.shift;
        dj.shift3 = sound ? jb.eps3 : 0;
        dj.T3 = 2 * dj.shift3;
        dj.shift2 = 0;
        if (sound) {
            uint64_t e2 = 0;
            const tmd_status s2 = sound_piece_eps(jb, jb.eps3, &e2);
            if (s2 != TMD_OK) return s2;
            dj.shift2 = e2;
        }
        dj.T2 = 2 * dj.shift2;
        dj.shift2s = 0;
        const uint64_t n2 = sound_piece_length(jb.log2_N);
        if (sound && n2 > 64) {
            uint64_t e2s = 0;
            const tmd_status s2 = sound_line_eps(jb, jb.eps3, (n2 + 31) / 32, &e2s);
            if (s2 != TMD_OK) return s2;
            dj.shift2s = e2s;
        }
        dj.T2s = 2 * dj.shift2s;
        dj.log2_N = jb.log2_N;
        dj.log2_T = jb.log2_T;
        dj.d = (uint32_t)jb.d;
        dj.L = jb.limbs;
        dj.m = (uint32_t)jb.m;
        dj.flags = jb.flags;
        dj.func = jb.func;
        dj.e_in = jb.e_in;
        dj.p = jb.p;
        const uint64_t T = 1ull << jb.log2_T, N = 1ull << jb.log2_N;
        const uint64_t SB = T >> jb.log2_N;  // sub-intervals of a full block
        dj.nu = choose_nu(jb, SB, nu_max);
        dj.ppb = (uint32_t)((SB + dj.nu - 1) / dj.nu);
        // the 2d+1 step-N difference words, then (sound mode) the d+1
        // Taylor coefficients of the exhaustive phase
        dj.words = (uint32_t)(((sound ? 3 : 2) * jb.d + (sound ? 2 : 1)) * jb.limbs);
        dj.n_seg = (uint32_t)segs.size();
        uint64_t nb = 0, ns = 0, np = 0;
        for (size_t k = 0; k < segs.size(); k++) {
            const uint64_t len = segs[k].j1 - segs[k].j0;
            const uint64_t nfull = len >> jb.log2_T, rest = len & (T - 1);
            const uint64_t nsub_last = (rest + N - 1) >> jb.log2_N;
            dj.seg_j0[k] = segs[k].j0;
            dj.seg_j1[k] = segs[k].j1;
            dj.seg_e_out[k] = segs[k].e_out;
            dj.seg_block0[k] = nb;
            dj.seg_sub0[k] = ns;
            dj.seg_packet0[k] = np;
            nb += nfull + (rest ? 1 : 0);
            ns += nfull * SB + nsub_last;
            np += nfull * dj.ppb + (nsub_last + dj.nu - 1) / dj.nu;
        }
        if (nblk_total + nb >= (1ull << 31)) return TMD_EUNSUPPORTED;
        dj.line_off = line;
        dj.n_lines = ns;
        dj.block_off = (uint32_t)nblk_total;
        dj.n_blocks = (uint32_t)nb;
        dj.packet_off = packet;
        dj.n_packets = np;
        dj.table_off = toff;
        P.jobs.push_back(dj);
        line += ns;
        packet += np;
        toff += nb * dj.words;
        nblk_total += nb;
        P.total_args += jb.count;
    }
    P.total_lines = line;
    P.table_words = toff;
    P.n_blocks = nblk_total;
    // tasks class by class, job by job (stable); a class is (limbs, degree,
    // kernel variant: general when the job uses Lefevre's filter or the
    // sound mode)
    uint64_t task = 0;
    for (uint32_t key = 0; key < 16 * (MAX_LIMBS + 1); key++) {
        const uint64_t first = task;
        uint32_t Lk = 0, Dk = 0;
        for (uint32_t j = 0; j < njobs; j++) {
            const DevJob& dj = P.jobs[j];
            const uint32_t g = general_variant(dj.flags, (int)dj.m, dj.log2_N) ? 1u : 0u;
            if ((dj.L * 8 + dj.d) * 2 + g != key) continue;
            P.class_jobs.push_back(j);
            P.class_task0.push_back(task);
            task += (dj.n_packets + 31) / 32;
            Lk = dj.L;
            Dk = dj.d;
        }
        if (task > first) P.classes.push_back(ClassRange{Lk, Dk, (key & 1) != 0, first, task - first});
    }
    P.n_tasks = task;
    if (!host_tables) return TMD_OK;
    // host mode: materialise blocks, tasks and tables with the same formulas
    P.blocks.resize(P.n_blocks);
    for (uint32_t j = 0; j < njobs; j++)
        for (uint64_t rb = 0; rb < P.jobs[j].n_blocks; rb++)
            P.blocks[P.jobs[j].block_off + rb] = block_record(P.jobs[j], j, rb);
    P.tasks.resize(P.n_tasks);
    for (size_t e = 0; e < P.class_jobs.size(); e++) {
        const uint32_t j = P.class_jobs[e];
        const uint64_t nt = (P.jobs[j].n_packets + 31) / 32;
        for (uint64_t k = 0; k < nt; k++) P.tasks[P.class_task0[e] + k] = task_record(P.jobs[j], j, k);
    }
    P.tables.assign(toff, 0);
    // the anchors of the jobs, then the tables block by block
    std::vector<Anchor> anchors(njobs);
    std::atomic<uint32_t> next_job(0);
    run_threads(std::min<unsigned>(host_threads(), njobs), [&]() {
        std::vector<Segment> sg;
        for (;;) {
            const uint32_t j = next_job.fetch_add(1);
            if (j >= njobs) break;
            sg.assign(seg_of[j].begin(), seg_of[j].begin() + nseg_of[j]);
            host_anchor(jobs[j], sg, &anchors[j]);
        }
    });
    std::atomic<uint64_t> next(0);
    std::atomic<int> bad(0);
    const uint64_t nblk = P.n_blocks;
    auto worker = [&]() {
        for (;;) {
            uint64_t b = next.fetch_add(16);
            if (b >= nblk) break;
            uint64_t e = std::min<uint64_t>(b + 16, nblk);
            for (; b < e; b++) {
                const DevBlock& db = P.blocks[b];
                BlockPlan bp;
                bp.start = db.start;
                bp.length = db.length;
                bp.first_sub = db.first_sub;
                bp.e_out = db.e_out;
                const tmd_job& bj = jobs[db.job];
                uint64_t* tw = &P.tables[db.table_off];
                uint64_t* cw = (bj.flags & TMD_SOUND) ? tw + (2 * bj.d + 1) * bj.limbs : nullptr;
                if (block_table(bj, bp, cw, tw, &anchors[db.job]) != TMD_OK)
                    bad.store(1);
            }
        }
    };
    run_threads((unsigned)std::min<uint64_t>(host_threads(), (nblk + 15) / 16), worker);
    return bad.load() ? TMD_EUNSUPPORTED : TMD_OK;
}

// Device layout of a plan: jobs | class jobs | class first tasks | blocks |
// tasks | table status | tables.  Without host tables only the first three
// sections are uploaded; the planning and table kernels write the rest.
struct Layout {
    size_t o_cjobs, o_ctask, o_blocks, o_tasks, o_status, o_tables, total, upload;
};

Layout plan_layout(const Plan& P) {
    Layout L;
    L.o_cjobs = align256(P.jobs.size() * sizeof(DevJob));
    L.o_ctask = align256(L.o_cjobs + P.class_jobs.size() * sizeof(uint32_t));
    L.o_blocks = align256(L.o_ctask + P.class_task0.size() * sizeof(uint64_t));
    L.o_tasks = align256(L.o_blocks + P.n_blocks * sizeof(DevBlock));
    L.o_status = align256(L.o_tasks + P.n_tasks * sizeof(DevTask));
    L.o_tables = align256(L.o_status + P.n_blocks * sizeof(uint32_t));
    L.total = align256(L.o_tables + P.table_words * sizeof(uint64_t));
    L.upload = P.host_tables ? L.total : L.o_blocks;
    return L;
}

void pack_plan(const Plan& P, const Layout& L, char* dst) {
    memset(dst, 0, L.upload);
    memcpy(dst, P.jobs.data(), P.jobs.size() * sizeof(DevJob));
    memcpy(dst + L.o_cjobs, P.class_jobs.data(), P.class_jobs.size() * sizeof(uint32_t));
    memcpy(dst + L.o_ctask, P.class_task0.data(), P.class_task0.size() * sizeof(uint64_t));
    if (P.host_tables) {
        memcpy(dst + L.o_blocks, P.blocks.data(), P.blocks.size() * sizeof(DevBlock));
        memcpy(dst + L.o_tasks, P.tasks.data(), P.tasks.size() * sizeof(DevTask));
        memcpy(dst + L.o_tables, P.tables.data(), P.tables.size() * sizeof(uint64_t));
    }
}

// after the upload: blocks, tasks and tables on the device (unless host mode)
// zero_misc / zero_count (optional): counters of the search that follows,
// cleared by the planning kernel (not when the tables came from the host:
// the caller clears them then).
// inl (optional): the uploaded words, passed to the planning kernel as its
// parameter instead of having been copied to d_arena.
cudaError_t expand_plan(const Plan& P, const Layout& L, char* d_arena, uint32_t* plan_err, const uint64_t* ctab,
                        cudaStream_t s, uint64_t* zero_misc = nullptr, uint32_t n_misc = 0,
                        uint64_t* zero_count = nullptr, const InlinePlan* inl = nullptr) {
    if (P.host_tables) return cudaSuccess;
    cudaError_t e =
        inl ? launch_plan_inline(*inl, (uint32_t)(L.upload / sizeof(uint64_t)), (uint64_t*)d_arena,
                                 (uint32_t)P.jobs.size(), L.o_cjobs, L.o_ctask, (uint32_t)P.class_jobs.size(),
                                 L.o_blocks, P.n_blocks, L.o_tasks, P.n_tasks, plan_err, zero_misc, n_misc, zero_count,
                                 s)
            : launch_plan((const DevJob*)d_arena, (uint32_t)P.jobs.size(), (DevBlock*)(d_arena + L.o_blocks),
                          P.n_blocks, (const uint32_t*)(d_arena + L.o_cjobs), (const uint64_t*)(d_arena + L.o_ctask),
                          (uint32_t)P.class_jobs.size(), (DevTask*)(d_arena + L.o_tasks), P.n_tasks, plan_err,
                          zero_misc, n_misc, zero_count, s);
    if (e != cudaSuccess) return e;
    uint32_t func_mask = 0;
    for (const DevJob& dj : P.jobs) func_mask |= 1u << (dj.func & 3);
    return launch_block_tables((const DevJob*)d_arena, (const DevBlock*)(d_arena + L.o_blocks), P.n_blocks,
                               (uint64_t*)(d_arena + L.o_tables), (uint32_t*)(d_arena + L.o_status), plan_err, ctab,
                               func_mask, s);
}

// Arena layout: jobs | class job lists | class first tasks | blocks | tasks |
// table status | tables.  The first three sections are uploaded (as the
// planning kernel's parameter when they fit in it); the tables are uploaded
// when they were made on the host, else written by the table kernel on the
// device.
tmd_status upload_plan(tmd_ctx* c, cudaStream_t s, uint64_t* zero_count, bool* zeroed) {
    Plan& P = c->plan;
    const Layout Lo = plan_layout(P);
    if (c->stage_pending) {
        CK(cudaEventSynchronize(c->stage_done));
        c->stage_pending = false;
    }
    if (Lo.upload > c->stage_cap) {
        if (c->h_stage) CK(cudaFreeHost(c->h_stage));
        c->h_stage = nullptr;
        size_t cap = std::max(Lo.upload, c->stage_cap * 2);
        CK(cudaHostAlloc((void**)&c->h_stage, cap, cudaHostAllocDefault));
        c->stage_cap = cap;
    }
    if (Lo.total > c->arena_cap) {
        CK(cudaStreamSynchronize(s));
        if (c->d_arena) CK(cudaFree(c->d_arena));
        c->d_arena = nullptr;
        size_t cap = std::max(Lo.total, c->arena_cap * 2);
        CK(cudaMalloc((void**)&c->d_arena, cap));
        c->arena_cap = cap;
    }
    // a small plan's records travel as the planning kernel's parameter (no
    // separate copy to wait for); larger ones through the pinned stage
    const bool inline_upload = !P.host_tables && Lo.upload <= sizeof(InlinePlan);
    InlinePlan inl;
    if (inline_upload) {
        pack_plan(P, Lo, (char*)inl.w);
    } else {
        pack_plan(P, Lo, c->h_stage);
        CK(cudaMemcpyAsync(c->d_arena, c->h_stage, Lo.upload, cudaMemcpyHostToDevice, s));
        CK(cudaEventRecord(c->stage_done, s));
        c->stage_pending = true;
    }
    c->upload_bytes = Lo.upload;
    c->off_jobs = 0;
    c->off_blocks = Lo.o_blocks;
    c->off_tables = Lo.o_tables;
    c->off_tasks = Lo.o_tasks;
    // the plan kernel clears the plan's error word; host-made tables have none
    if (P.host_tables) CK(cudaMemsetAsync(plan_err_ptr(c), 0, sizeof(uint32_t), s));
    const bool z = zeroed && !P.host_tables;
    CK(expand_plan(P, Lo, c->d_arena, plan_err_ptr(c), c->d_ctab, s, z ? c->d_misc : nullptr, z ? ST_COUNT + 1 : 0,
                   z ? zero_count : nullptr, inline_upload ? &inl : nullptr));
    if (zeroed) *zeroed = z;
    return TMD_OK;
}

bool same_jobs(const tmd_ctx* c, const tmd_job* jobs, uint32_t njobs) {
    if (!c->resident || c->plan.key.size() != njobs) return false;
    return memcmp(c->plan.key.data(), jobs, njobs * sizeof(tmd_job)) == 0;
}

// zeroed (optional): set when the planning kernel also cleared the search
// counters and *zero_count (a fresh plan made on the device)
tmd_status make_resident(tmd_ctx* c, const tmd_job* jobs, uint32_t njobs, cudaStream_t s,
                         uint64_t* zero_count = nullptr, bool* zeroed = nullptr) {
    if (zeroed) *zeroed = false;
    if (same_jobs(c, jobs, njobs)) return TMD_OK;
    c->resident = false;
    tmd_status st = build_plan(jobs, njobs, c->plan, /*host_tables=*/false);
    if (st != TMD_OK) return st;
    st = upload_plan(c, s, zero_count, zeroed);
    if (st != TMD_OK) return st;
    c->resident = true;
    return TMD_OK;
}

LaunchArgs task_args(tmd_ctx* c) {
    LaunchArgs a;
    memset(&a, 0, sizeof a);
    a.jobs = (const DevJob*)(c->d_arena + c->off_jobs);
    a.blocks = (const DevBlock*)(c->d_arena + c->off_blocks);
    a.tables = (const uint64_t*)(c->d_arena + c->off_tables);
    a.tasks = (const DevTask*)(c->d_arena + c->off_tasks);
    a.n_tasks = c->plan.n_tasks;
    a.stats = stats_ptr(c);
    a.queue_head = queue_ptr(c);
    return a;
}

tmd_status reset_counters(tmd_ctx* c, uint64_t* d_count, cudaStream_t s) {
    CK(launch_zero_counters(c->d_misc, ST_COUNT + 1, d_count, s));
    return TMD_OK;
}

}  // namespace

extern "C" {

const char* tmd_version(void) { return "tmd-gb300 0.1 (sm_103a)"; }

const char* tmd_status_str(tmd_status s) {
    switch (s) {
        case TMD_OK: return "ok";
        case TMD_EINVAL: return "invalid argument";
        case TMD_ENOMEM: return "buffer too small or allocation failed";
        case TMD_EOVERFLOW: return "candidate capacity exceeded (count is exact)";
        case TMD_ETIMEOUT: return "bounded device wait expired";
        case TMD_ECUDA: return "CUDA runtime error";
        case TMD_EUNSUPPORTED: return "unsupported by this build";
    }
    return "unknown status";
}

tmd_status tmd_create(tmd_ctx** out, int device) {
    if (!out) return TMD_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return TMD_ECUDA;
    CK(cudaSetDevice(device));
    tmd_ctx* c = new tmd_ctx();
    c->device = device;
    if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMalloc((void**)&c->d_misc, 64) != cudaSuccess ||
        cudaHostAlloc((void**)&c->h_small, 64, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&c->d_small, c->h_small, 0) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->stage_done, cudaEventDisableTiming) != cudaSuccess) {
        tmd_destroy(c);
        return TMD_ECUDA;
    }
    cudaMemset(c->d_misc, 0, 64);
    if (upload_coeff_consts(coeff_consts()) != cudaSuccess) {
        tmd_destroy(c);
        return TMD_ECUDA;
    }
    // the exp and 2^x tables of the block-table kernel, built once per context
    uint32_t terr = 0;
    if (cudaMalloc((void**)&c->d_ctab, CT_WORDS * sizeof(uint64_t)) != cudaSuccess ||
        launch_coeff_tables(c->d_ctab, plan_err_ptr(c), nullptr) != cudaSuccess ||
        cudaMemcpy(&terr, plan_err_ptr(c), sizeof terr, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(plan_err_ptr(c), 0, sizeof(uint32_t)) != cudaSuccess) {
        tmd_destroy(c);
        return TMD_ECUDA;
    }
    if (terr) {
        tmd_destroy(c);
        return TMD_EUNSUPPORTED;
    }
    *out = c;
    return TMD_OK;
}

tmd_status tmd_destroy(tmd_ctx* c) {
    if (!c) return TMD_EINVAL;
    cudaSetDevice(c->device);
    if (c->stage_pending) cudaEventSynchronize(c->stage_done);
    if (c->d_arena) cudaFree(c->d_arena);
    if (c->d_misc) cudaFree(c->d_misc);
    if (c->d_ctab) cudaFree(c->d_ctab);
    if (c->h_stage) cudaFreeHost(c->h_stage);
    if (c->h_small) cudaFreeHost(c->h_small);
    if (c->stage_done) cudaEventDestroy(c->stage_done);
    delete c;
    return TMD_OK;
}

tmd_status tmd_evict(tmd_ctx* c) {
    if (!c) return TMD_EINVAL;
    c->resident = false;
    c->plan.key.clear();
    return TMD_OK;
}

tmd_status tmd_plan(const tmd_job* job, tmd_plan_info* info) {
    if (!job || !info) return TMD_EINVAL;
    tmd_status st = validate_job(*job);
    if (st != TMD_OK) return st;
    std::vector<Segment> segs;
    st = plan_segments(*job, segs);
    if (st != TMD_OK) return st;
    memset(info, 0, sizeof *info);
    plan_counts(*job, segs, &info->n_blocks, &info->n_subints);
    info->n_segments = (uint32_t)segs.size();
    info->e_out_first = segs[0].e_out;
    for (size_t i = 1; i < segs.size() && i <= 4; i++) info->cut[i - 1] = segs[i].j0;
    return TMD_OK;
}

tmd_status tmd_sound_eps(const tmd_job* job, uint64_t* eps1, uint64_t* eps3) {
    if (!job || !eps1 || !eps3) return TMD_EINVAL;
    return sound_eps(*job, eps1, eps3);
}

tmd_status tmd_sound_line_eps(const tmd_job* job, uint64_t length, uint64_t* eps) {
    if (!job || !eps) return TMD_EINVAL;
    return sound_line_eps(*job, job->eps3, length, eps);
}

tmd_status tmd_sound_piece_eps(const tmd_job* job, uint64_t* eps2) {
    if (!job || !eps2) return TMD_EINVAL;
    return sound_piece_eps(*job, job->eps3, eps2);
}

tmd_status tmd_block_tables(const tmd_job* job, uint64_t block, uint64_t* coeffs, uint64_t* table,
                            tmd_block_info* info) {
    if (!job) return TMD_EINVAL;
    tmd_status st = validate_job(*job);
    if (st != TMD_OK) return st;
    std::vector<Segment> segs;
    st = plan_segments(*job, segs);
    if (st != TMD_OK) return st;
    BlockPlan bp;
    if (!plan_block(*job, segs, block, &bp)) return TMD_EINVAL;
    if (info) {
        info->start = bp.start;
        info->length = bp.length;
        info->first_sub = bp.first_sub;
        info->e_out = bp.e_out;
        info->scale_log2 = scale_log2(*job, bp.e_out);
    }
    Anchor A;
    host_anchor(*job, segs, &A);
    return block_table(*job, bp, coeffs, table, &A);
}

tmd_status tmd_generate(tmd_ctx* c, const tmd_job* jobs, uint32_t njobs, void* d_lin, size_t lin_bytes,
                        size_t* lin_bytes_needed, void* stream) {
    if (!c || !jobs || njobs == 0) return TMD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(c->device));
    tmd_status st = make_resident(c, jobs, njobs, s);
    if (st != TMD_OK) return st;
    const size_t need = (size_t)c->plan.total_lines * 16;
    if (lin_bytes_needed) *lin_bytes_needed = need;
    if (!d_lin) return TMD_OK;
    if (lin_bytes < need) return TMD_ENOMEM;
    LaunchArgs base = task_args(c);
    base.lin_B = (uint64_t*)d_lin;
    base.lin_A = (uint64_t*)d_lin + c->plan.total_lines;
    for (const ClassRange& cr : c->plan.classes) {
        LaunchArgs a = base;
        a.tasks = base.tasks + cr.first;
        a.n_tasks = cr.count;
        CK(launch_tasks(false, cr.L, cr.D, cr.G, a, s));
    }
    return TMD_OK;
}

tmd_status tmd_search(tmd_ctx* c, const tmd_job* jobs, uint32_t njobs, const void* d_lin,
                      tmd_candidate* d_cand, uint64_t cand_cap, uint64_t* d_count, void* stream) {
    if (!c || !jobs || njobs == 0 || !d_count || (cand_cap && !d_cand)) return TMD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(c->device));
    bool zeroed = false;
    tmd_status st = make_resident(c, jobs, njobs, s, d_count, &zeroed);
    if (st != TMD_OK) return st;
    if (!zeroed) {
        st = reset_counters(c, d_count, s);
        if (st != TMD_OK) return st;
    }
    c->last_count = d_count;
    if (d_lin) {
        LineArgs a;
        memset(&a, 0, sizeof a);
        a.B = (const uint64_t*)d_lin;
        a.A = (const uint64_t*)d_lin + c->plan.total_lines;
        a.n_lines = c->plan.total_lines;
        a.jobs = (const DevJob*)(c->d_arena + c->off_jobs);
        a.n_jobs = (uint32_t)c->plan.jobs.size();
        a.blocks = (const DevBlock*)(c->d_arena + c->off_blocks);
        a.tables = (const uint64_t*)(c->d_arena + c->off_tables);
        a.cand = d_cand;
        a.cap = cand_cap;
        a.count = d_count;
        a.stats = stats_ptr(c);
        a.err = err_ptr(c);
        CK(launch_search_lines(false, a, s));
        return TMD_OK;
    }
    LaunchArgs base = task_args(c);
    base.cand = d_cand;
    base.cap = cand_cap;
    base.count = d_count;
    for (const ClassRange& cr : c->plan.classes) {
        LaunchArgs a = base;
        a.tasks = base.tasks + cr.first;
        a.n_tasks = cr.count;
        CK(launch_tasks(true, cr.L, cr.D, cr.G, a, s));
    }
    return TMD_OK;
}

tmd_status tmd_candidates(tmd_ctx* c, const tmd_candidate* d_cand, const uint64_t* d_count,
                          uint64_t cand_cap, tmd_candidate* h_out, uint64_t h_cap, uint64_t* n_out,
                          void* stream) {
    if (!c || !d_count || !n_out || (h_cap && !h_out)) return TMD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(c->device));
    // one small kernel writes the count and the error words into mapped
    // host memory, then one wait (copies to pageable memory would each wait
    // for the stream)
    volatile uint64_t* hs = c->h_small;
    CK(launch_readback(d_count, err_ptr(c), c->d_small, s));
    CK(cudaStreamSynchronize(s));
    const uint64_t count = hs[0];
    const uint32_t err = (uint32_t)hs[1], perr = (uint32_t)hs[2];  // hs[1] >> 32: the queue head
    if (perr) return TMD_EUNSUPPORTED;
    *n_out = count;
    uint64_t n = std::min(count, std::min(cand_cap, h_cap));
    if (n) {
        if (!d_cand) return TMD_EINVAL;
        CK(cudaMemcpyAsync(h_out, d_cand, n * sizeof(tmd_candidate), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        std::sort(h_out, h_out + n, [](const tmd_candidate& a, const tmd_candidate& b) {
            if (a.job != b.job) return a.job < b.job;
            if (a.arg_index != b.arg_index) return a.arg_index < b.arg_index;
            return a.value < b.value;
        });
    }
    if (err) return TMD_EINVAL;
    return count > n ? TMD_EOVERFLOW : TMD_OK;
}

tmd_status tmd_search_lines(tmd_ctx* c, const uint64_t* d_B, const uint64_t* d_A, const uint32_t* d_len,
                            uint64_t n, int32_t m, uint32_t flags, tmd_candidate* d_cand,
                            uint64_t cand_cap, uint64_t* d_count, void* stream) {
    if (!c || !d_count || (n && (!d_B || !d_A || !d_len)) || (cand_cap && !d_cand)) return TMD_EINVAL;
    if (m < 2 || m > 63 || (flags & ~(uint32_t)(TMD_ALL_HITS | TMD_LEFEVRE))) return TMD_EINVAL;
    if (n >= (1ull << 32)) return TMD_EUNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(c->device));
    tmd_status st = reset_counters(c, d_count, s);
    if (st != TMD_OK) return st;
    c->last_count = d_count;
    LineArgs a;
    memset(&a, 0, sizeof a);
    a.B = d_B;
    a.A = d_A;
    a.len = d_len;
    a.n_lines = n;
    a.Tm = 1ull << (65 - m);
    a.flags = flags;
    a.cand = d_cand;
    a.cap = cand_cap;
    a.count = d_count;
    a.stats = stats_ptr(c);
    a.err = err_ptr(c);
    CK(launch_search_lines(true, a, s));
    return TMD_OK;
}

tmd_status tmd_lower_bounds(tmd_ctx* c, const uint64_t* d_B, const uint64_t* d_A, const uint32_t* d_len,
                            uint64_t n, uint64_t* d_lb, uint32_t* d_hs, void* stream) {
    if (!c || (n && (!d_B || !d_A || !d_len || !d_lb))) return TMD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(c->device));
    CK(cudaMemsetAsync(err_ptr(c), 0, sizeof(uint32_t), s));
    CK(launch_lower_bounds(0, d_B, d_A, d_len, n, d_lb, d_hs, err_ptr(c), s));
    return TMD_OK;
}

tmd_status tmd_lefevre_bounds(tmd_ctx* c, const uint64_t* d_B, const uint64_t* d_A, const uint32_t* d_len,
                              uint64_t n, uint32_t specific, uint64_t* d_lb, uint32_t* d_iters, void* stream) {
    if (!c || (n && (!d_B || !d_A || !d_len || !d_lb)) || specific > 1) return TMD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(c->device));
    CK(cudaMemsetAsync(err_ptr(c), 0, sizeof(uint32_t), s));
    CK(launch_lower_bounds(specific ? 2 : 1, d_B, d_A, d_len, n, d_lb, d_iters, err_ptr(c), s));
    return TMD_OK;
}

tmd_status tmd_stats_read(tmd_ctx* c, tmd_stats* out, void* stream) {
    if (!c || !out) return TMD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(c->device));
    uint64_t h[ST_COUNT];
    uint64_t cnt = 0;
    CK(cudaMemcpyAsync(h, stats_ptr(c), sizeof h, cudaMemcpyDeviceToHost, s));
    if (c->last_count) CK(cudaMemcpyAsync(&cnt, c->last_count, sizeof cnt, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    out->lines = h[ST_LINES];
    out->filter_fail = h[ST_FAIL];
    out->candidates = cnt;
    out->half_steps = h[ST_HALF];
    out->upload_bytes = c->upload_bytes;
    out->count = cnt;
    out->exhaustive_args = h[ST_EXH];
    out->refined_args = h[ST_REF];
    return TMD_OK;
}

// ---------------------------------------------------------------- batches
}  // extern "C"

// batch counters: stats[5] | error | unused | plan error | pad | queue heads (one per class)
enum { BATCH_MISC_BYTES = 192, BATCH_QUEUE_OFF = 64 };

struct tmd_batch {
    tmd_ctx* ctx = nullptr;
    Plan plan;
    char* d_arena = nullptr;
    uint64_t* d_misc = nullptr;
    size_t off_jobs = 0, off_blocks = 0, off_tables = 0, off_tasks = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    uint64_t upload_bytes = 0;
    const uint64_t* d_count = nullptr;
    tmd_tiling tiling = {0, 0, 0, 0};
};

namespace {

void batch_free(tmd_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->d_arena) cudaFree(b->d_arena);
    if (b->d_misc) cudaFree(b->d_misc);
    delete b;
}

// Signature of a batch for the tuned-tiling cache: its distinct (limbs,
// degree, log2 N) classes, the SM count and the order of magnitude of its
// sub-interval count (the tiling decides how the tasks divide among the
// resident warps, so the size matters).
std::string tiling_key(const tmd_job* jobs, uint32_t njobs, int sms) {
    std::vector<uint32_t> cls;
    double subs = 0;
    for (uint32_t j = 0; j < njobs; j++) {
        cls.push_back(jobs[j].limbs * 1024u + (uint32_t)jobs[j].d * 32u + jobs[j].log2_N);
        subs += (double)((jobs[j].count + (1ull << jobs[j].log2_N) - 1) >> jobs[j].log2_N);
    }
    std::sort(cls.begin(), cls.end());
    cls.erase(std::unique(cls.begin(), cls.end()), cls.end());
    std::string k = "sms" + std::to_string(sms) + "/subs2^" + std::to_string((int)std::log2(std::max(subs, 1.0)));
    for (uint32_t v : cls)
        k += "/L" + std::to_string(v >> 10) + "d" + std::to_string((v >> 5) & 31) + "N" + std::to_string(v & 31);
    return k;
}

tmd_status batch_create(tmd_ctx* c, const tmd_job* jobs, uint32_t njobs, tmd_candidate* d_cand,
                        uint64_t cand_cap, uint64_t* d_count, void* stream, const tmd_tiling& tiling,
                        tmd_batch** out, uint64_t* upload_bytes);

}  // namespace

extern "C" {

tmd_status tmd_batch_create(tmd_ctx* c, const tmd_job* jobs, uint32_t njobs, tmd_candidate* d_cand,
                            uint64_t cand_cap, uint64_t* d_count, void* stream, tmd_batch** out,
                            uint64_t* upload_bytes) {
    if (!c || !jobs || njobs == 0 || !d_count || !out || (cand_cap && !d_cand)) return TMD_EINVAL;
    tmd_tiling t = {0, 0, 0, 0};
    {
        std::lock_guard<std::mutex> lk(c->tune_mu);
        auto it = c->tuned.find(tiling_key(jobs, njobs, c->sms));
        if (it != c->tuned.end()) t = it->second;
    }
    return batch_create(c, jobs, njobs, d_cand, cand_cap, d_count, stream, t, out, upload_bytes);
}

tmd_status tmd_batch_create_tiled(tmd_ctx* c, const tmd_job* jobs, uint32_t njobs, tmd_candidate* d_cand,
                                  uint64_t cand_cap, uint64_t* d_count, void* stream, const tmd_tiling* tiling,
                                  tmd_batch** out, uint64_t* upload_bytes) {
    if (!c || !jobs || njobs == 0 || !d_count || !out || (cand_cap && !d_cand)) return TMD_EINVAL;
    tmd_tiling t = tiling ? *tiling : tmd_tiling{0, 0, 0, 0};
    if (t.nu > 8 || t.ctas_per_sm > 64 || t.lanes == 3 || t.lanes > 4 || t.unroll > 2) return TMD_EINVAL;
    return batch_create(c, jobs, njobs, d_cand, cand_cap, d_count, stream, t, out, upload_bytes);
}

tmd_status tmd_autotune(tmd_ctx* c, const tmd_job* jobs, uint32_t njobs, void* stream, tmd_tiling* best,
                        float* best_ms) {
    if (!c || !jobs || njobs == 0 || !best) return TMD_EINVAL;
    CK(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    // the largest occupancy over the batch's classes bounds the CTA counts tried
    int occ = 1;
    for (uint32_t j = 0; j < njobs; j++) {
        int per_sm = 0;
        if (jobs[j].limbs >= 1 && jobs[j].limbs <= 3 && jobs[j].d >= 1 && jobs[j].d <= 4 &&
            persistent_occupancy(jobs[j].limbs, (uint32_t)jobs[j].d,
                                 general_variant(jobs[j].flags, jobs[j].m, jobs[j].log2_N),
                                 &per_sm) == cudaSuccess)
            occ = std::max(occ, per_sm);
    }
    uint64_t* d_cnt = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc((void**)&d_cnt, sizeof(uint64_t)) != cudaSuccess) return TMD_ENOMEM;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaFree(d_cnt);
        if (e0) cudaEventDestroy(e0);
        return TMD_ECUDA;
    }
    tmd_status st = TMD_OK;
    // mean replay time of the batch under tiling t (one warm replay first)
    auto time_tiling = [&](const tmd_tiling& t, int reps, float* out) -> tmd_status {
        tmd_batch* b = nullptr;
        tmd_status s2 = batch_create(c, jobs, njobs, nullptr, 0, d_cnt, stream, t, &b, nullptr);
        if (s2 != TMD_OK) return s2;
        float ms = 0.f;
        if (cudaGraphLaunch(b->exec, s) != cudaSuccess || cudaEventRecord(e0, s) != cudaSuccess) s2 = TMD_ECUDA;
        for (int r = 0; r < reps && s2 == TMD_OK; r++)
            if (cudaGraphLaunch(b->exec, s) != cudaSuccess) s2 = TMD_ECUDA;
        if (s2 == TMD_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            s2 = TMD_ECUDA;
        tmd_batch_destroy(b);
        *out = ms / (float)reps;
        return s2;
    };
    // stage 1: packet length x resident CTAs (one lane per line, one step
    // per iteration); stage 2: lanes per line x steps per iteration for the
    // stage-1 winner; then the three fastest of all are timed again with
    // more replays (single timings of a few replays differ by ~1-3 %)
    std::vector<tmd_tiling> cands;
    std::vector<float> times;
    static const uint32_t nus[] = {8, 6, 4, 2, 1};
    for (uint32_t nu : nus)
        for (int k = occ; k >= 1; k--) cands.push_back(tmd_tiling{nu, (uint32_t)k, 1, 1});
    const size_t stage1 = cands.size();
    for (size_t ci = 0; ci < cands.size() && st == TMD_OK; ci++) {
        if (ci == stage1) {
            const size_t w = (size_t)(std::min_element(times.begin(), times.end()) - times.begin());
            static const uint32_t lanes_unroll[][2] = {{1, 2}, {2, 1}, {2, 2}, {4, 1}, {4, 2}};
            for (const auto& lu : lanes_unroll)
                cands.push_back(tmd_tiling{cands[w].nu, cands[w].ctas_per_sm, lu[0], lu[1]});
        }
        float ms = 0.f;
        st = time_tiling(cands[ci], 4, &ms);
        times.push_back(ms);
    }
    tmd_tiling win = {0, 0, 0, 0};
    float win_ms = 0.f;
    if (st == TMD_OK) {
        std::vector<size_t> order(cands.size());
        for (size_t i = 0; i < order.size(); i++) order[i] = i;
        std::sort(order.begin(), order.end(), [&](size_t x, size_t y) { return times[x] < times[y]; });
        for (size_t r = 0; r < std::min<size_t>(3, order.size()) && st == TMD_OK; r++) {
            float ms = 0.f;
            st = time_tiling(cands[order[r]], 16, &ms);
            if (st == TMD_OK && (win.nu == 0 || ms < win_ms)) {
                win = cands[order[r]];
                win_ms = ms;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d_cnt);
    if (st != TMD_OK) return st;
    {
        std::lock_guard<std::mutex> lk(c->tune_mu);
        c->tuned[tiling_key(jobs, njobs, c->sms)] = win;
    }
    *best = win;
    if (best_ms) *best_ms = win_ms;
    return TMD_OK;
}

}  // extern "C"

namespace {

tmd_status batch_create(tmd_ctx* c, const tmd_job* jobs, uint32_t njobs, tmd_candidate* d_cand,
                        uint64_t cand_cap, uint64_t* d_count, void* stream, const tmd_tiling& tiling,
                        tmd_batch** out, uint64_t* upload_bytes) {
    *out = nullptr;
    CK(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    tmd_batch* b = new tmd_batch();
    b->ctx = c;
    b->d_count = d_count;
    b->tiling = tiling;
    tmd_status st = build_plan(jobs, njobs, b->plan, /*host_tables=*/false, tiling.nu);
    if (st != TMD_OK) {
        batch_free(b);
        return st;
    }
    Plan& P = b->plan;
    b->tiling.nu = 0;
    for (const DevJob& dj : P.jobs) b->tiling.nu = std::max(b->tiling.nu, dj.nu);
    b->tiling.ctas_per_sm = 0;
    const Layout Lo = plan_layout(P);
    const size_t o_blocks = Lo.o_blocks, o_tasks = Lo.o_tasks, o_tables = Lo.o_tables;
    std::vector<char> host(Lo.upload, 0);
    pack_plan(P, Lo, host.data());
    uint32_t* plan_err = nullptr;
    uint32_t perr = 0;
    if (cudaMalloc((void**)&b->d_arena, Lo.total) != cudaSuccess ||
        cudaMalloc((void**)&b->d_misc, BATCH_MISC_BYTES) != cudaSuccess ||
        cudaMemsetAsync(b->d_misc, 0, BATCH_MISC_BYTES, s) != cudaSuccess ||
        cudaMemcpyAsync(b->d_arena, host.data(), Lo.upload, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        batch_free(b);
        return TMD_ECUDA;
    }
    plan_err = (uint32_t*)(b->d_misc + ST_COUNT) + 2;
    if (expand_plan(P, Lo, b->d_arena, plan_err, c->d_ctab, s) != cudaSuccess ||
        cudaMemcpyAsync(&perr, plan_err, sizeof perr, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        batch_free(b);
        return TMD_ECUDA;
    }
    if (perr) {
        batch_free(b);
        return TMD_EUNSUPPORTED;
    }
    b->upload_bytes = Lo.upload;
    if (upload_bytes) *upload_bytes = Lo.upload;
    b->off_blocks = o_blocks;
    b->off_tables = o_tables;
    b->off_tasks = o_tasks;
    // one persistent launch per (limbs, degree) class, each over its own task
    // range with its own queue head; grid = every SM filled to the kernel's
    // occupancy, no more CTAs than the class's tasks need
    LaunchArgs a;
    memset(&a, 0, sizeof a);
    a.jobs = (const DevJob*)b->d_arena;
    a.blocks = (const DevBlock*)(b->d_arena + o_blocks);
    a.tables = (const uint64_t*)(b->d_arena + o_tables);
    a.cand = d_cand;
    a.cap = cand_cap;
    a.count = d_count;
    a.stats = b->d_misc;
    a.lanes = tiling.lanes;
    a.unroll = tiling.unroll;
    b->tiling.lanes = tiling.lanes ? tiling.lanes : 1;
    b->tiling.unroll = tiling.unroll ? tiling.unroll : 1;
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        batch_free(b);
        return TMD_ECUDA;
    }
    cudaMemsetAsync(b->d_misc, 0, BATCH_MISC_BYTES, b->cap_stream);
    cudaMemsetAsync(d_count, 0, sizeof(uint64_t), b->cap_stream);
    static_assert(BATCH_QUEUE_OFF + 4 * 3 * 4 * 2 <= BATCH_MISC_BYTES, "one queue head per class");
    if (P.classes.size() > 24) {
        cudaStreamEndCapture(b->cap_stream, &b->graph);
        batch_free(b);
        return TMD_EUNSUPPORTED;
    }
    for (size_t ci = 0; ci < P.classes.size(); ci++) {
        const ClassRange& cr = P.classes[ci];
        int per_sm = 0;
        if (persistent_occupancy(cr.L, cr.D, cr.G, &per_sm) != cudaSuccess || per_sm < 1) per_sm = 1;
        if (tiling.ctas_per_sm) per_sm = std::min(per_sm, (int)tiling.ctas_per_sm);
        b->tiling.ctas_per_sm = std::max(b->tiling.ctas_per_sm, (uint32_t)per_sm);
        const uint64_t want = (cr.count + 7) / 8;
        const int ctas = (int)std::min<uint64_t>((uint64_t)c->sms * (uint64_t)per_sm, std::max<uint64_t>(want, 1));
        LaunchArgs ac = a;
        ac.tasks = (const DevTask*)(b->d_arena + o_tasks) + cr.first;
        ac.n_tasks = cr.count;
        ac.queue_head = (uint32_t*)((char*)b->d_misc + BATCH_QUEUE_OFF) + ci;  // ci < 24: inside the 192 B
        launch_persistent(cr.L, cr.D, cr.G, ac, ctas, b->cap_stream);
    }
    if (cudaStreamEndCapture(b->cap_stream, &b->graph) != cudaSuccess ||
        cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) {
        batch_free(b);
        return TMD_ECUDA;
    }
    *out = b;
    return TMD_OK;
}

}  // namespace

extern "C" {

tmd_status tmd_batch_tiling(const tmd_batch* b, tmd_tiling* out) {
    if (!b || !out) return TMD_EINVAL;
    *out = b->tiling;
    return TMD_OK;
}

tmd_status tmd_batch_launch(tmd_batch* b, void* stream) {
    if (!b) return TMD_EINVAL;
    CK(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    return TMD_OK;
}

tmd_status tmd_batch_stats(tmd_batch* b, tmd_stats* out, void* stream) {
    if (!b || !out) return TMD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t h[ST_COUNT];
    uint64_t cnt = 0;
    CK(cudaMemcpyAsync(h, b->d_misc, sizeof h, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&cnt, b->d_count, sizeof cnt, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    out->lines = h[ST_LINES];
    out->filter_fail = h[ST_FAIL];
    out->candidates = cnt;
    out->half_steps = h[ST_HALF];
    out->upload_bytes = b->upload_bytes;
    out->count = cnt;
    out->exhaustive_args = h[ST_EXH];
    out->refined_args = h[ST_REF];
    return TMD_OK;
}

tmd_status tmd_batch_destroy(tmd_batch* b) {
    if (!b) return TMD_EINVAL;
    cudaSetDevice(b->ctx->device);
    batch_free(b);
    return TMD_OK;
}

}  // extern "C"

// ------------------------------------------------------------ serving loop
//
// Continuous batching.  A host worker thread admits the jobs that have
// arrived (in arrival order, up to max_batch at a time, while their plans fit
// the device budget) into a free slot as one group: it plans the group on the
// host, uploads its job records and enqueues on the slot's stream the device
// planning, the correctly rounded tables, one fused search launch per kernel
// class and the read-back of the group's count.  A stream callback hands the
// slot back to the worker, which reads the records (if any) and splits them
// into per-job results.  While one group runs on the device the worker plans
// and launches the next in another slot, and the fused launches of the slots
// share the SMs.  Jobs may be submitted with an arrival time in the future
// (tmd_server_submit_many), so that a recorded or generated arrival stream is
// replayed by the server's clock without a host loop in between.

namespace {

struct ServerJob {
    tmd_job job;
    uint64_t id;
    double t_submit;  // arrival time on the server clock
    size_t est;       // plan bytes estimate (for the device budget)
    bool solo;        // re-run alone after its group overflowed the records
};

struct ServerResult {
    tmd_job_result r;
    std::vector<tmd_candidate> recs;
};

// Slot meta block on the device: stats[5] | error | queue head | plan error | pad | count.
enum { META_BYTES = 128, META_COUNT_OFF = 64 };

// One resident group of jobs: its stream, plan arena, records and counters.
struct Slot {
    enum State { FREE, RUNNING, READING };
    cudaStream_t stream = nullptr;
    char* d_arena = nullptr;
    size_t arena_cap = 0;
    tmd_candidate* d_cand = nullptr;
    char* d_meta = nullptr;
    char* h_stage = nullptr;
    size_t stage_cap = 0;
    char* h_meta = nullptr;          // pinned copy of the meta block
    tmd_candidate* h_recs = nullptr;  // pinned records (cand_cap)
    State state = FREE;
    std::vector<ServerJob> sjs;
    std::vector<tmd_job> jobs;
    double t_start = 0;
    Plan plan;
    size_t plan_bytes = 0;
    uint64_t count = 0, n_read = 0;
    tmd_status status = TMD_OK;
    // stream-callback argument (stable address: slots are never resized)
    void* server = nullptr;
    int index = 0;
};

}  // namespace

struct tmd_server {
    tmd_ctx* ctx = nullptr;
    tmd_server_config cfg;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ServerJob> pending;                 // arrived, in arrival order
    std::multimap<double, ServerJob> future;       // arrival time -> job
    std::deque<int> events;                        // slots whose stream reached a callback
    std::deque<ServerResult> finished;
    std::vector<Slot> slots;
    size_t budget_used = 0;
    uint64_t outstanding = 0;
    bool stop = false;
    std::chrono::steady_clock::time_point t0;
    // totals over the finished groups (tmd_server_stats)
    uint64_t st_lines = 0, st_fail = 0, st_half = 0, st_exh = 0, st_ref = 0, st_groups = 0, st_count = 0;
};

namespace {

double server_now(const tmd_server* S) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - S->t0).count();
}

size_t plan_estimate(const tmd_job& job) {
    uint64_t nb = 0, ns = 0;
    std::vector<Segment> segs;
    if (plan_segments(job, segs) == TMD_OK) plan_counts(job, segs, &nb, &ns);
    return (size_t)nb * (sizeof(DevBlock) + 4 + (size_t)(2 * job.d + 1) * job.limbs * 8) +
           (size_t)(ns / 8 / 32 + nb + 1) * sizeof(DevTask) + 4096;
}

void CUDART_CB slot_callback(void* arg) {
    Slot* sl = (Slot*)arg;
    tmd_server* S = (tmd_server*)sl->server;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->events.push_back(sl->index);
    }
    S->cv_work.notify_one();
}

// plan, upload, device planning and tables, fused search launches and the
// read-back of the meta block of a group, all enqueued on the slot's stream
tmd_status slot_start(tmd_server* S, Slot& sl) {
    sl.t_start = server_now(S);
    sl.jobs.clear();
    for (const ServerJob& sj : sl.sjs) sl.jobs.push_back(sj.job);
    tmd_status st = build_plan(sl.jobs.data(), (uint32_t)sl.jobs.size(), sl.plan, /*host_tables=*/false);
    if (st != TMD_OK) return st;
    Plan& P = sl.plan;
    const Layout Lo = plan_layout(P);
    if (Lo.total > sl.arena_cap) {
        if (sl.d_arena) CK(cudaFreeAsync(sl.d_arena, sl.stream));
        sl.d_arena = nullptr;
        const size_t cap = std::max(Lo.total, sl.arena_cap + sl.arena_cap / 2);
        CK(cudaMallocAsync((void**)&sl.d_arena, cap, sl.stream));
        sl.arena_cap = cap;
    }
    if (Lo.upload > sl.stage_cap) {
        CK(cudaStreamSynchronize(sl.stream));
        if (sl.h_stage) CK(cudaFreeHost(sl.h_stage));
        sl.h_stage = nullptr;
        const size_t cap = std::max(Lo.upload, sl.stage_cap * 2);
        CK(cudaHostAlloc((void**)&sl.h_stage, cap, cudaHostAllocDefault));
        sl.stage_cap = cap;
    }
    pack_plan(P, Lo, sl.h_stage);
    CK(cudaMemcpyAsync(sl.d_arena, sl.h_stage, Lo.upload, cudaMemcpyHostToDevice, sl.stream));
    CK(cudaMemsetAsync(sl.d_meta, 0, META_BYTES, sl.stream));
    uint32_t* perr = (uint32_t*)(sl.d_meta + sizeof(uint64_t) * ST_COUNT) + 2;
    CK(expand_plan(P, Lo, sl.d_arena, perr, S->ctx->d_ctab, sl.stream));
    LaunchArgs a;
    memset(&a, 0, sizeof a);
    a.jobs = (const DevJob*)sl.d_arena;
    a.blocks = (const DevBlock*)(sl.d_arena + Lo.o_blocks);
    a.tables = (const uint64_t*)(sl.d_arena + Lo.o_tables);
    a.cand = sl.d_cand;
    a.cap = S->cfg.cand_cap;
    a.count = (uint64_t*)(sl.d_meta + META_COUNT_OFF);
    a.stats = (uint64_t*)sl.d_meta;
    a.queue_head = (uint32_t*)(sl.d_meta + sizeof(uint64_t) * ST_COUNT) + 1;
    const uint64_t chunk = S->cfg.chunk_tasks ? S->cfg.chunk_tasks : ~0ull;
    for (const ClassRange& cr : P.classes) {
        for (uint64_t pos = 0; pos < cr.count; pos += chunk) {
            LaunchArgs la = a;
            la.tasks = (const DevTask*)(sl.d_arena + Lo.o_tasks) + cr.first + pos;
            la.n_tasks = std::min<uint64_t>(chunk, cr.count - pos);
            CK(launch_tasks(true, cr.L, cr.D, cr.G, la, sl.stream));
        }
    }
    CK(cudaMemcpyAsync(sl.h_meta, sl.d_meta, META_BYTES, cudaMemcpyDeviceToHost, sl.stream));
    CK(cudaLaunchHostFunc(sl.stream, slot_callback, &sl));
    sl.state = Slot::RUNNING;
    return TMD_OK;
}

void slot_release(tmd_server* S, Slot& sl) {
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->budget_used -= sl.plan_bytes;
    }
    sl.state = Slot::FREE;
    sl.sjs.clear();
    sl.plan_bytes = 0;
}

// the group's results, split per job; a group whose records overflowed goes
// back to the queue front job by job
void slot_finish(tmd_server* S, Slot& sl) {
    const double t_done = server_now(S);
    tmd_status st = sl.status;
    const uint64_t count = sl.count;
    const bool overflow = st == TMD_OK && count > S->cfg.cand_cap;
    if (overflow && sl.sjs.size() > 1) {
        std::vector<ServerJob> again = sl.sjs;
        slot_release(S, sl);
        std::lock_guard<std::mutex> lk(S->mu);
        for (size_t k = again.size(); k-- > 0;) {
            again[k].solo = true;
            S->pending.push_front(again[k]);
        }
        return;
    }
    std::vector<tmd_candidate> recs(sl.h_recs, sl.h_recs + (st == TMD_OK ? sl.n_read : 0));
    std::sort(recs.begin(), recs.end(), [](const tmd_candidate& a, const tmd_candidate& b) {
        if (a.job != b.job) return a.job < b.job;
        if (a.arg_index != b.arg_index) return a.arg_index < b.arg_index;
        return a.value < b.value;
    });
    std::vector<ServerResult> out(sl.sjs.size());
    size_t pos = 0;
    for (size_t k = 0; k < sl.sjs.size(); k++) {
        ServerResult& R = out[k];
        memset(&R.r, 0, sizeof R.r);
        R.r.id = sl.sjs[k].id;
        R.r.t_submit = sl.sjs[k].t_submit;
        R.r.t_start = sl.t_start;
        R.r.t_done = t_done;
        while (pos < recs.size() && recs[pos].job == k) {
            tmd_candidate c = recs[pos++];
            c.job = 0;  // as the job's own run reports it
            R.recs.push_back(c);
        }
        R.r.count = overflow ? count : R.recs.size();
        R.r.n_records = R.recs.size();
        R.r.status = st == TMD_OK ? (overflow ? TMD_EOVERFLOW : TMD_OK) : st;
    }
    slot_release(S, sl);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (ServerResult& R : out) S->finished.push_back(std::move(R));
    }
    S->cv_done.notify_all();
}

// a slot's stream reached its callback: the meta block (count, counters,
// plan error) is on the host, or, in the READING state, the records
void slot_event(tmd_server* S, Slot& sl) {
    if (sl.state == Slot::RUNNING) {
        const uint64_t* h = (const uint64_t*)sl.h_meta;
        const uint32_t* err = (const uint32_t*)(sl.h_meta + sizeof(uint64_t) * ST_COUNT);
        sl.count = *(const uint64_t*)(sl.h_meta + META_COUNT_OFF);
        sl.status = err[2] ? TMD_EUNSUPPORTED : TMD_OK;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->st_lines += h[ST_LINES];
            S->st_fail += h[ST_FAIL];
            S->st_half += h[ST_HALF];
            S->st_exh += h[ST_EXH];
            S->st_ref += h[ST_REF];
            S->st_groups += 1;
            S->st_count += sl.count;
        }
        const bool rerun = sl.status == TMD_OK && sl.count > S->cfg.cand_cap && sl.sjs.size() > 1;
        sl.n_read = sl.status == TMD_OK && !rerun ? std::min<uint64_t>(sl.count, S->cfg.cand_cap) : 0;
        if (sl.n_read) {
            if (cudaMemcpyAsync(sl.h_recs, sl.d_cand, sl.n_read * sizeof(tmd_candidate), cudaMemcpyDeviceToHost,
                                sl.stream) != cudaSuccess ||
                cudaLaunchHostFunc(sl.stream, slot_callback, &sl) != cudaSuccess) {
                cudaStreamSynchronize(sl.stream);
                sl.status = TMD_ECUDA;
                slot_finish(S, sl);
                return;
            }
            sl.state = Slot::READING;
            return;
        }
    }
    slot_finish(S, sl);
}

void server_loop(tmd_server* S) {
    cudaSetDevice(S->ctx->device);
    std::vector<int> evs;
    for (;;) {
        evs.clear();
        bool any_busy = false;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            const double now = server_now(S);
            while (!S->future.empty() && S->future.begin()->first <= now) {
                S->pending.push_back(S->future.begin()->second);
                S->future.erase(S->future.begin());
            }
            evs.assign(S->events.begin(), S->events.end());
            S->events.clear();
            for (const Slot& sl : S->slots) any_busy |= sl.state != Slot::FREE;
            if (S->stop) {
                S->pending.clear();
                S->future.clear();
                if (!any_busy && evs.empty()) break;
            }
        }
        bool progress = !evs.empty();
        for (int i : evs) slot_event(S, S->slots[(size_t)i]);
        // admission: the oldest arrived jobs, up to max_batch, while they fit
        for (Slot& sl : S->slots) {
            if (sl.state != Slot::FREE) continue;
            size_t take = 0, bytes = 0;
            {
                std::unique_lock<std::mutex> lk(S->mu);
                if (S->pending.empty()) break;
                while (take < S->pending.size() && take < S->cfg.max_batch) {
                    const ServerJob& sj = S->pending[take];
                    if (take > 0 && (sj.solo || S->pending[0].solo)) break;
                    if ((S->budget_used > 0 || take > 0) && S->budget_used + bytes + sj.est > S->cfg.device_budget)
                        break;
                    bytes += sj.est;
                    take++;
                }
                if (take == 0) break;
                sl.sjs.assign(S->pending.begin(), S->pending.begin() + (long)take);
                S->pending.erase(S->pending.begin(), S->pending.begin() + (long)take);
                S->budget_used += bytes;
            }
            sl.plan_bytes = bytes;
            sl.status = TMD_OK;
            sl.count = sl.n_read = 0;
            if (slot_start(S, sl) != TMD_OK) {
                cudaStreamSynchronize(sl.stream);
                sl.status = TMD_ECUDA;
                slot_finish(S, sl);
            }
            progress = true;
        }
        if (progress) continue;
        std::unique_lock<std::mutex> lk(S->mu);
        if (!S->events.empty()) continue;
        if (S->stop) {
            if (any_busy) S->cv_work.wait_for(lk, std::chrono::milliseconds(50));
            continue;
        }
        bool can_admit = !S->pending.empty();
        if (can_admit) {
            can_admit = false;
            for (const Slot& sl : S->slots) can_admit |= sl.state == Slot::FREE;
        }
        if (can_admit) continue;
        // sleep until a callback, a submission, or the next scheduled arrival
        double wait_s = 0.05;
        if (!S->future.empty()) wait_s = std::min(wait_s, std::max(0.0, S->future.begin()->first - server_now(S)));
        if (wait_s > 0)
            S->cv_work.wait_for(lk, std::chrono::duration<double>(wait_s));
    }
}

}  // namespace

extern "C" {

tmd_status tmd_server_create(tmd_ctx* c, const tmd_server_config* cfg, tmd_server** out) {
    if (!c || !out) return TMD_EINVAL;
    *out = nullptr;
    tmd_server_config k;
    memset(&k, 0, sizeof k);
    if (cfg) k = *cfg;
    if (k.reserved != 0) return TMD_EINVAL;
    if (k.device_budget == 0) k.device_budget = 1ull << 30;
    if (k.max_inflight == 0) k.max_inflight = 4;
    if (k.cand_cap == 0) k.cand_cap = 65536;
    if (k.max_batch == 0) k.max_batch = 1024;
    if (k.max_inflight > 64) return TMD_EINVAL;
    CK(cudaSetDevice(c->device));
    tmd_server* S = new tmd_server();
    S->ctx = c;
    S->cfg = k;
    S->t0 = std::chrono::steady_clock::now();
    S->slots.resize(k.max_inflight);
    for (size_t i = 0; i < S->slots.size(); i++) {
        Slot& sl = S->slots[i];
        sl.server = S;
        sl.index = (int)i;
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMalloc((void**)&sl.d_cand, k.cand_cap * sizeof(tmd_candidate)) != cudaSuccess ||
            cudaMalloc((void**)&sl.d_meta, META_BYTES) != cudaSuccess ||
            cudaHostAlloc((void**)&sl.h_meta, META_BYTES, cudaHostAllocDefault) != cudaSuccess ||
            cudaHostAlloc((void**)&sl.h_recs, k.cand_cap * sizeof(tmd_candidate), cudaHostAllocDefault) !=
                cudaSuccess) {
            tmd_server_destroy(S);
            return TMD_ECUDA;
        }
    }
    S->worker = std::thread(server_loop, S);
    *out = S;
    return TMD_OK;
}

tmd_status tmd_server_submit(tmd_server* S, const tmd_job* job, uint64_t id) {
    if (!S || !job) return TMD_EINVAL;
    tmd_status st = validate_job(*job);
    if (st != TMD_OK) return st;
    const size_t est = plan_estimate(*job);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return TMD_EINVAL;
        S->pending.push_back(ServerJob{*job, id, server_now(S), est, false});
        S->outstanding++;
    }
    S->cv_work.notify_one();
    return TMD_OK;
}

tmd_status tmd_server_submit_many(tmd_server* S, const tmd_job* jobs, const uint64_t* ids,
                                  const double* delays_s, uint32_t n) {
    if (!S || (n && (!jobs || !ids || !delays_s))) return TMD_EINVAL;
    std::vector<size_t> est(n);
    for (uint32_t i = 0; i < n; i++) {
        if (!(delays_s[i] >= 0.0)) return TMD_EINVAL;
        tmd_status st = validate_job(jobs[i]);
        if (st != TMD_OK) return st;
        est[i] = plan_estimate(jobs[i]);
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return TMD_EINVAL;
        const double now = server_now(S);
        for (uint32_t i = 0; i < n; i++) {
            const double t = now + delays_s[i];
            S->future.emplace(t, ServerJob{jobs[i], ids[i], t, est[i], false});
        }
        S->outstanding += n;
    }
    S->cv_work.notify_one();
    return TMD_OK;
}

tmd_status tmd_server_poll(tmd_server* S, tmd_job_result* out, uint32_t cap, uint32_t* n_out,
                           tmd_candidate* h_records, uint64_t rec_cap, uint64_t* rec_out, int32_t wait_ms) {
    if (!S || !n_out || (cap && !out) || (rec_cap && !h_records)) return TMD_EINVAL;
    *n_out = 0;
    if (rec_out) *rec_out = 0;
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->finished.empty() && wait_ms > 0)
        S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !S->finished.empty(); });
    uint64_t used = 0;
    uint32_t n = 0;
    while (n < cap && !S->finished.empty()) {
        ServerResult& R = S->finished.front();
        const uint64_t take = std::min<uint64_t>(R.recs.size(), rec_cap - used);
        if (take) memcpy(h_records + used, R.recs.data(), take * sizeof(tmd_candidate));
        used += take;
        out[n] = R.r;
        out[n].n_records = take;
        n++;
        S->finished.pop_front();
        S->outstanding--;
    }
    *n_out = n;
    if (rec_out) *rec_out = used;
    return TMD_OK;
}

tmd_status tmd_server_pending(tmd_server* S, uint64_t* n) {
    if (!S || !n) return TMD_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    *n = S->outstanding;
    return TMD_OK;
}

tmd_status tmd_server_stats(tmd_server* S, tmd_stats* out, uint64_t* groups) {
    if (!S || !out) return TMD_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    memset(out, 0, sizeof *out);
    out->lines = S->st_lines;
    out->filter_fail = S->st_fail;
    out->candidates = S->st_count;
    out->half_steps = S->st_half;
    out->count = S->st_count;
    out->exhaustive_args = S->st_exh;
    out->refined_args = S->st_ref;
    if (groups) *groups = S->st_groups;
    return TMD_OK;
}

double tmd_server_clock(tmd_server* S) { return S ? server_now(S) : 0.0; }

tmd_status tmd_server_destroy(tmd_server* S) {
    if (!S) return TMD_EINVAL;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->ctx->device);
    for (Slot& sl : S->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.d_arena) cudaFreeAsync(sl.d_arena, sl.stream);
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.d_cand) cudaFree(sl.d_cand);
        if (sl.d_meta) cudaFree(sl.d_meta);
        if (sl.h_stage) cudaFreeHost(sl.h_stage);
        if (sl.h_meta) cudaFreeHost(sl.h_meta);
        if (sl.h_recs) cudaFreeHost(sl.h_recs);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    delete S;
    return TMD_OK;
}

}  // extern "C"

// ------------------------------------------------- no-allocation entry point
// tmd_search_static keeps everything the search needs besides the caller's
// inputs and outputs -- the plan arena (jobs, blocks, tables, work list) and
// the counters -- in one file-scope device array instead of memory from
// cudaMalloc.  The array exists on every device that loads the library until
// the process exits.  Host code must not pass `g_static_scratch` itself to a
// kernel (in host code that name is a host-side stand-in); its device address
// is taken once per device with cudaGetSymbolAddress and cached below.

namespace {

constexpr size_t STATIC_MISC_BYTES = 256;  // stats[5], error word, queue head
__device__ __align__(256) unsigned char g_static_scratch[STATIC_MISC_BYTES + TMD_STATIC_SCRATCH_BYTES];

constexpr int STATIC_MAX_DEVICES = 64;
std::mutex g_static_mutex;
char* g_static_base[STATIC_MAX_DEVICES] = {};

// Device address of the scratch array on the current device (set-up on the
// first call per device).  The address belongs to the device's primary
// context: after cudaDeviceReset the cached value is stale.
tmd_status static_scratch_base(int device, char** out) {
    if (device < 0 || device >= STATIC_MAX_DEVICES) return TMD_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_base[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || p == nullptr) return TMD_ECUDA;
        g_static_base[device] = (char*)p;
    }
    *out = g_static_base[device];
    return TMD_OK;
}

}  // namespace

extern "C" {

tmd_status tmd_search_static(const tmd_job* jobs, uint32_t njobs, tmd_candidate* d_cand,
                             uint64_t cand_cap, uint64_t* d_count, void* stream) {
    if (!jobs || njobs == 0 || !d_count || (cand_cap && !d_cand)) return TMD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    // the plan goes up from a host buffer that lives only for this call: a
    // capturing stream would keep a copy node that reads it on every replay
    cudaStreamCaptureStatus cap_st = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &cap_st));
    if (cap_st != cudaStreamCaptureStatusNone) return TMD_EUNSUPPORTED;
    int device = 0;
    CK(cudaGetDevice(&device));
    char* base = nullptr;
    tmd_status st = static_scratch_base(device, &base);
    if (st != TMD_OK) return st;
    // sizes first (counts and offsets only), so that an oversized plan is
    // refused before any correctly rounded table is computed
    Plan P;
    st = build_plan(jobs, njobs, P, /*host_tables=*/false);
    if (st != TMD_OK) return st;
    const size_t o_blocks = align256(P.jobs.size() * sizeof(DevJob));
    const size_t o_tables = align256(o_blocks + P.n_blocks * sizeof(DevBlock));
    const size_t o_tasks = align256(o_tables + P.table_words * sizeof(uint64_t));
    const size_t total = align256(o_tasks + P.n_tasks * sizeof(DevTask));
    if (total > TMD_STATIC_SCRATCH_BYTES) return TMD_ENOMEM;
    st = build_plan(jobs, njobs, P, /*host_tables=*/true);
    if (st != TMD_OK) return st;
    std::vector<char> host(total, 0);
    memcpy(host.data(), P.jobs.data(), P.jobs.size() * sizeof(DevJob));
    memcpy(host.data() + o_blocks, P.blocks.data(), P.blocks.size() * sizeof(DevBlock));
    memcpy(host.data() + o_tables, P.tables.data(), P.tables.size() * sizeof(uint64_t));
    memcpy(host.data() + o_tasks, P.tasks.data(), P.tasks.size() * sizeof(DevTask));
    char* arena = base + STATIC_MISC_BYTES;
    // pageable source: the call returns once the bytes are staged, so the
    // vector may go out of scope afterwards
    CK(cudaMemcpyAsync(arena, host.data(), total, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(base, 0, STATIC_MISC_BYTES, s));
    CK(cudaMemsetAsync(d_count, 0, sizeof(uint64_t), s));
    LaunchArgs a;
    memset(&a, 0, sizeof a);
    a.jobs = (const DevJob*)arena;
    a.blocks = (const DevBlock*)(arena + o_blocks);
    a.tables = (const uint64_t*)(arena + o_tables);
    a.tasks = (const DevTask*)(arena + o_tasks);
    a.cand = d_cand;
    a.cap = cand_cap;
    a.count = d_count;
    a.stats = (uint64_t*)base;
    a.queue_head = (uint32_t*)(base + sizeof(uint64_t) * ST_COUNT) + 1;
    for (const ClassRange& cr : P.classes) {
        LaunchArgs la = a;
        la.tasks = a.tasks + cr.first;
        la.n_tasks = cr.count;
        CK(launch_tasks(true, cr.L, cr.D, cr.G, la, s));
    }
    return TMD_OK;
}

}  // extern "C"
