// Device-visible plan records (written by the host layer, read by kernels).
#pragma once

#include <cstdint>

#include "../../include/tmd.h"

namespace tmd {

// One job as the kernels see it.
struct DevJob {
    uint64_t line_off;     // global index of the job's first line (unfused layout)
    uint64_t n_lines;      // sub-intervals of the job
    uint64_t Tm;           // threshold 2^(65-m) on the search words
    uint32_t block_off;    // global index of the job's first block
    uint32_t n_blocks;
    uint32_t log2_N;
    uint32_t d;
    uint32_t L;            // limbs of the fixed-point words
    uint32_t m;
    uint32_t flags;
    uint32_t nu;           // sub-intervals per packet (lane)
    int32_t func;          // tmd_func
    int32_t e_in;
    int32_t p;
    uint32_t n_seg;        // output-binade segments (1..4)
    // device-side planning: the job's blocks and packets, segment by segment
    uint64_t packet_off;   // global index of the job's first packet
    uint64_t n_packets;
    uint64_t table_off;    // word offset of the job's first block table
    uint32_t ppb;          // packets of a full block
    uint32_t words;        // table words of a block ((2d+1) L)
    uint64_t seg_j0[4];    // first argument of each segment
    uint64_t seg_j1[4];    // end of each segment
    uint64_t seg_block0[4];    // job-relative first block of each segment
    uint64_t seg_sub0[4];      // job-relative first sub-interval of each segment
    uint64_t seg_packet0[4];   // job-relative first packet of each segment
    int32_t seg_e_out[4];
    uint32_t log2_T;
    uint32_t pad;
    uint64_t shift;        // added to the top word of b: 2^(64-m), or eps1 in sound mode (Tm = 2 shift)
    uint64_t shift3;       // sound mode: the exhaustive phase's half-width eps3 (T3 = 2 eps3)
    uint64_t T3;
    uint64_t shift2;       // sound mode: the phase-2 pieces' half-width eps2 (T2 = 2 eps2)
    uint64_t T2;
    uint64_t shift2s;      // sound mode: half-width of the pieces' 32 sub-pieces (0: pieces of
    uint64_t T2s;          // at most 64 arguments go to the exhaustive phase directly)
};

// One Taylor block.
struct DevBlock {
    uint64_t start;        // argument index of the first argument
    uint64_t length;       // arguments in the block
    uint64_t first_sub;    // job-wide index of the first sub-interval
    uint64_t packet_off;   // global index of the block's first packet
    uint64_t table_off;    // offset (in 64-bit words) of the block's 2d+1 table words
    uint32_t job;
    uint32_t n_sub;        // sub-intervals in the block
    int32_t e_out;         // output exponent on the block
    uint32_t pad;
};

// A warp's unit of work: up to 32 consecutive packets of one job.
struct DevTask {
    uint64_t g0;           // first global packet index
    uint32_t count;        // packets (1..32)
    uint32_t job;
    uint32_t block0;       // global index of the block holding packet g0
    uint32_t pad;
};

// Error bits of the context's error word.
enum { ERR_BAD_LENGTH = 1, ERR_ROUNDING = 2 };

// Counters (device uint64 each) in the order of tmd_stats.
// ST_EXH: arguments evaluated one by one in the sound mode; ST_REF: arguments
// of the phase-2 pieces the sound mode keeps (phase 3's input)
enum { ST_LINES = 0, ST_FAIL = 1, ST_EXH = 2, ST_HALF = 3, ST_REF = 4, ST_COUNT = 5 };

// Launch-side description of one fused/unfused launch.
// The uploaded part of a small plan (job records, class lists) passed by
// value as the planning kernel's parameter (3 KB, under the classic 4 KB
// limit of kernel parameters) instead of a host-to-device copy.
constexpr int INLINE_PLAN_WORDS = 384;
struct InlinePlan {
    uint64_t w[INLINE_PLAN_WORDS];
};

struct LaunchArgs {
    const DevJob* jobs;
    const DevBlock* blocks;
    const uint64_t* tables;
    const DevTask* tasks;
    uint64_t n_tasks;
    uint64_t* lin_B;        // unfused layout: B[total lines], A[total lines]
    uint64_t* lin_A;
    tmd_candidate* cand;
    uint64_t cap;
    uint64_t* count;
    uint64_t* stats;
    uint32_t* queue_head;   // persistent form: next task index
    uint32_t lanes;         // lanes per line in the filter (0, 1: one; 2; 4)
    uint32_t unroll;        // difference steps per iteration of the stepping loop (0, 1: one; 2)
};

// Line search arguments.  JOBS mode: the lines written by the generation
// kernel for the resident plan.  RAW mode: caller arrays with lengths.
struct LineArgs {
    const uint64_t* B;
    const uint64_t* A;
    const uint32_t* len;      // RAW only
    uint64_t n_lines;
    uint64_t Tm;              // RAW only
    uint32_t flags;           // RAW only
    const DevJob* jobs;       // JOBS only
    uint32_t n_jobs;
    const DevBlock* blocks;
    const uint64_t* tables;   // JOBS only: the block tables (sound jobs' phases 2 and 3)
    tmd_candidate* cand;
    uint64_t cap;
    uint64_t* count;
    uint64_t* stats;
    uint32_t* err;
};

}  // namespace tmd
