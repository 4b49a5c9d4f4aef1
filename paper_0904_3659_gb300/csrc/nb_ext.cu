// nb_ext.cu -- context-owned buffers of the other entry points.
#include "nb_ext.h"

namespace nbx {

void ext_release(ExtState &s) {
    for (int k = 0; k < ExtState::kSlots; ++k) {
        cudaFree(s.buf[k]);
        s.buf[k] = nullptr;
        s.cap[k] = 0;
    }
}

}  // namespace nbx
