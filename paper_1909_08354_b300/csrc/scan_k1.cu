// The batched scan's kernel at a register budget of 1 resident CTA per SM
// (scan_kernel.cuh), in a translation unit of its own.
#include "scan_kernel.cuh"

namespace sn_scan {
ScanKern scan_kernel_1() { return scan_kernel<1>; }
}  // namespace sn_scan
