// Kernel (a)'s instances for packed relation rows (RAC_LAYOUT_PACKED, layout
// codes 16 + q): the same kernel source compiled as a second translation unit,
// which defines launch_bits_packed instead of launch_bits, so that the
// library's two largest sets of instances compile in parallel.
#define RAC_BITS_PACKED_UNIT
#include "rac_bits_kernel.cu"
