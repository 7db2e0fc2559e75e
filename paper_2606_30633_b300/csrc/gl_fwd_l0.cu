// k_forward instantiations with 0 lens-light component(s).
#include "gl_fwd_impl.cuh"

namespace gl {
GL_FWD_INST(, 0)
}  // namespace gl
