// Pencil FFT passes instantiated for transform length 288 (144-point grids).
#include "passes.cuh"
namespace lsgpu {
LS_DEFINE_LENGTH(288)
}  // namespace lsgpu
