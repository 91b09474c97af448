// Host-side planning and block tables (shared by the C-ABI layer).
#pragma once

#include <cstdint>
#include <vector>

#include "../../include/tmd.h"

namespace tmd {

enum { MAX_LIMBS = 3, MAX_DEG = 4, MAX_WORDS = 2 * MAX_DEG + 1, MAX_SEGMENTS = 4 };

struct Segment {
    uint64_t j0, j1;   // [j0, j1) argument indices
    int e_out;
};

struct BlockPlan {
    uint64_t start, length, first_sub;
    int e_out;
};

// Validation of one job (domain of this build); TMD_OK when usable.
tmd_status validate_job(const tmd_job& job);
// The sound thresholds (eps1, eps3) of a job, on the 64-bit words.
tmd_status sound_eps(const tmd_job& job, uint64_t* eps1, uint64_t* eps3);
// Arguments of a phase-2 piece (a sub-interval is cut into 32) and the
// phase-2 half-width for a sound job's eps3.
uint32_t sound_piece_length(uint32_t log2_N);
tmd_status sound_piece_eps(const tmd_job& job, uint64_t eps3, uint64_t* eps2);
tmd_status sound_line_eps(const tmd_job& job, uint64_t eps3, uint64_t length, uint64_t* eps);

// e(f(X_j)) (Def. 1) for argument index j.
int output_exponent(const tmd_job& job, uint64_t j);

// Output-binade segments of the job's slice (cuts decided exactly).
tmd_status plan_segments(const tmd_job& job, std::vector<Segment>& segs);

// Number of blocks / sub-intervals of a job from its segments.
void plan_counts(const tmd_job& job, const std::vector<Segment>& segs,
                 uint64_t* n_blocks, uint64_t* n_subints);

// The block with plan index b (0-based).  Returns false past the end.
bool plan_block(const tmd_job& job, const std::vector<Segment>& segs, uint64_t b,
                BlockPlan* out);

// log2 of the breakpoint scale s on a segment with output exponent e_out.
int scale_log2(const tmd_job& job, int e_out);

struct Anchor;
// Enclosure of f at the job's first argument, at the precision of its first
// segment (A->ok = 0 when it cannot be formed or the job has one block).
void host_anchor(const tmd_job& job, const std::vector<Segment>& segs, Anchor* A);

// Coefficients c_0..c_d (limbs each, little-endian) and the 2d+1 table words
// of the block, from the job's anchor when given.  TMD_EUNSUPPORTED if the
// rounding could not be decided.
tmd_status block_table(const tmd_job& job, const BlockPlan& blk, uint64_t* coeffs,
                       uint64_t* table, const Anchor* anchor = nullptr);

struct CoeffConsts;
// Constants of the coefficient routine (divisor reciprocals, ln 2), computed
// once per process.
const CoeffConsts& coeff_consts();

}  // namespace tmd
