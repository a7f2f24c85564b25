// NNDSVD initialisation from compressed data (Boutsidis & Gallopoulos 2008).
#include "common.cuh"

namespace nmfrp {

size_t nndsvd_ws_bytes(int64_t, int64_t, int, int) { return 256; }

cudaError_t launch_nndsvd(const Launcher&, int64_t, int64_t, int, int, const float*, const float*,
                          float*, float*, void*, size_t, int*) {
  return cudaErrorNotSupported;
}

}  // namespace nmfrp
