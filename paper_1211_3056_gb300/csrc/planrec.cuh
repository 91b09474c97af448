// Block and task records of a plan from its per-job segment table, shared by
// the host planner and the device planning kernels (same formulas on both).
//
// Within a segment [j0, j1) of one output exponent the blocks start at j0 and
// hold T arguments (the last one less); a block's sub-intervals are split into
// packets of nu (ppb packets for a full block, fewer for the last); a task is
// 32 consecutive packets of one job.
#pragma once

#include "dev.hpp"
#include "fxp.cuh"

namespace tmd {

TMD_HD uint32_t job_segment_of_block(const DevJob& J, uint64_t rb) {
    uint32_t sg = 0;
    for (uint32_t k = 1; k < J.n_seg; k++)
        if (J.seg_block0[k] <= rb) sg = k;
    return sg;
}

TMD_HD uint32_t job_segment_of_packet(const DevJob& J, uint64_t rp) {
    uint32_t sg = 0;
    for (uint32_t k = 1; k < J.n_seg; k++)
        if (J.seg_packet0[k] <= rp) sg = k;
    return sg;
}

// block rb (job-relative) of job j
TMD_HD DevBlock block_record(const DevJob& J, uint32_t j, uint64_t rb) {
    const uint32_t sg = job_segment_of_block(J, rb);
    const uint64_t bis = rb - J.seg_block0[sg];
    const uint64_t T = 1ull << J.log2_T;
    DevBlock db;
    db.start = J.seg_j0[sg] + bis * T;
    const uint64_t left = J.seg_j1[sg] - db.start;
    db.length = left < T ? left : T;
    db.first_sub = J.seg_sub0[sg] + (bis << (J.log2_T - J.log2_N));
    db.packet_off = J.packet_off + J.seg_packet0[sg] + bis * J.ppb;
    db.table_off = J.table_off + rb * J.words;
    db.job = j;
    db.n_sub = (uint32_t)((db.length + (1ull << J.log2_N) - 1) >> J.log2_N);
    db.e_out = J.seg_e_out[sg];
    db.pad = 0;
    return db;
}

// task k (job-relative) of job j
TMD_HD DevTask task_record(const DevJob& J, uint32_t j, uint64_t k) {
    const uint64_t rp = k * 32;
    const uint32_t sg = job_segment_of_packet(J, rp);
    DevTask dt;
    dt.g0 = J.packet_off + rp;
    const uint64_t left = J.n_packets - rp;
    dt.count = (uint32_t)(left < 32 ? left : 32);
    dt.job = j;
    dt.block0 = J.block_off + (uint32_t)(J.seg_block0[sg] + (rp - J.seg_packet0[sg]) / J.ppb);
    dt.pad = 0;
    return dt;
}

}  // namespace tmd
