// Tuned parameters of the batched sort, per array-size class: the keys per
// sub-bucket aimed at by the first range split of an array.  Written by
// paper_2107_03290_gb300/autotune.py (the sweep and the GPU it ran on are in
// the comment below); edit by re-running it, not by hand.
//
// NVIDIA GB300, 2026-12-04: ls_sort_batch_ex on the batched
// workload's arrays of each class, median ms per call:
//   class 0 (1948 arrays, 66320707 keys): 512: 4.021, 768: 4.072, 1024: 4.063, 1536: 4.041, 2048: 4.068, 2560: 4.096, 3072: 4.213, 4096: 4.252
//   class 1 (1901 arrays, 320226495 keys): 512: 12.152, 768: 12.402, 1024: 12.202, 1536: 12.431, 2048: 12.559, 2560: 13.436, 3072: 13.598, 4096: 14.053
//   class 2 (132 arrays, 114713439 keys): 512: 4.334, 768: 4.306, 1024: 4.271, 1536: 4.376, 2048: 4.345, 2560: 4.654, 3072: 4.715, 4096: 4.832
#pragma once
#include <stdint.h>

namespace ls {
constexpr uint32_t TUNED_CLASS_MAX[3] = {65536u, 524288u, 0xFFFFFFFFu};  // largest array per class
constexpr uint32_t TUNED_SPLIT_TARGET[3] = {512u, 512u, 1024u};
}  // namespace ls
