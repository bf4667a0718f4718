// The batched scan's kernel at a register budget of 2 resident CTAs per SM
// (scan_kernel.cuh), in a translation unit of its own.
#include "scan_kernel.cuh"

namespace sn_scan {
ScanKern scan_kernel_2() { return scan_kernel<2>; }
}  // namespace sn_scan
