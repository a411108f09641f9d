// Tuned parameters of the batched sort, per array-size class: the keys per
// sub-bucket aimed at by the first range split of an array.  Written by
// paper_2107_03290_gb300/autotune.py (the sweep and the GPU it ran on are in
// the comment below); edit by re-running it, not by hand.
//
// NVIDIA GB300, 2026-12-04: ls_sort_batch_ex on the batched
// workload's arrays of each class, median ms per call:
//   class 0 (1948 arrays, 66320707 keys): 1024: 4.344, 1536: 4.284, 2048: 4.220, 2560: 4.314, 3072: 4.418, 3584: 4.437, 4096: 4.448, 6144: 4.564
//   class 1 (1901 arrays, 320226495 keys): 1024: 12.606, 1536: 12.633, 2048: 12.769, 2560: 13.648, 3072: 13.800, 3584: 14.037, 4096: 14.225, 6144: 14.723
//   class 2 (132 arrays, 114713439 keys): 1024: 4.309, 1536: 4.397, 2048: 4.369, 2560: 4.664, 3072: 4.756, 3584: 4.801, 4096: 4.867, 6144: 5.000
#pragma once
#include <stdint.h>

namespace ls {
constexpr uint32_t TUNED_CLASS_MAX[3] = {65536u, 524288u, 0xFFFFFFFFu};  // largest array per class
constexpr uint32_t TUNED_SPLIT_TARGET[3] = {2048u, 1024u, 1024u};
}  // namespace ls
