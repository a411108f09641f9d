// Tuned parameters of the batched sort, per array-size class: the keys per
// sub-bucket aimed at by the first range split of an array.  Written by
// paper_2107_03290_gb300/autotune.py (the sweep and the GPU it ran on are in
// the comment below); edit by re-running it, not by hand.
//
// NVIDIA GB300, 2026-12-04: ls_sort_batch_ex on the batched
// workload's arrays of each class, median ms per call:
//   class 0 (1948 arrays, 66320707 keys): 512: 3.971, 768: 4.049, 1024: 4.016, 1536: 4.010, 2048: 4.024, 2560: 4.030, 3072: 4.158, 4096: 4.222
//     (a sampled RMI per array instead, ls_sort on each: 473.9 ms)
//   class 1 (1901 arrays, 320226495 keys): 512: 11.991, 768: 12.160, 1024: 12.044, 1536: 12.258, 2048: 12.337, 2560: 13.151, 3072: 13.363, 4096: 13.932
//     (a sampled RMI per array instead, ls_sort on each: 518.6 ms)
//   class 2 (132 arrays, 114713439 keys): 512: 4.349, 768: 4.320, 1024: 4.293, 1536: 4.412, 2048: 4.390, 2560: 4.601, 3072: 4.740, 4096: 4.889
//     (a sampled RMI per array instead, ls_sort on each: 46.6 ms)
#pragma once
#include <stdint.h>

namespace ls {
constexpr uint32_t TUNED_CLASS_MAX[3] = {65536u, 524288u, 0xFFFFFFFFu};  // largest array per class
constexpr uint32_t TUNED_SPLIT_TARGET[3] = {512u, 512u, 1024u};
}  // namespace ls
