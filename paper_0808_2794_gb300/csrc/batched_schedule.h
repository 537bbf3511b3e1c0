// batched_schedule.h -- panel width of the batched solver's FP32 factorization
// per range of n, as chosen by the autotuner (paper_0808_2794_gb300/tune_batched.py,
// which times every candidate width on each range of the batch of 4096 systems
// and rewrites this file).  Entry i covers kBatchedNmax[i-1] < n <= kBatchedNmax[i].
// Tuned 2026-12-04 on NVIDIA GB300: milliseconds per launch of the range's systems
// for panel widths 8, 16:
//   n in (0, 32]: 864 systems: 0.834, 0.850 -> 8
//   n in (32, 64]: 804 systems: 1.339, 1.353 -> 8
//   n in (64, 128]: 830 systems: 2.417, 2.412 -> 16
//   n in (128, 256]: 783 systems: 4.714, 4.626 -> 16
//   n in (256, 512]: 815 systems: 13.532, 12.503 -> 16
#pragma once
static const int kBatchedRanges = 5;
static const int kBatchedNmax[kBatchedRanges] = {32, 64, 128, 256, 512};
static const int kBatchedNb[kBatchedRanges] = {8, 8, 16, 16, 16};
