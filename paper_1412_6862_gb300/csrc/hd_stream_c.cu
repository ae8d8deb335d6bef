// hd_stream_c.cu -- compiled streaming-decoder configurations for n = 127, 255.
#include "hd_stream.cuh"

namespace hd {

void register_stream_c(std::vector<StreamVariant> &v)
{
    add_variants<127, 128, 3, 16, 1>(v);
    add_variants<127, 64, 4, 16, 1>(v);
    add_variants<127, 256, 3, 8, 1>(v);
    add_variants<127, 128, 4, 8, 1>(v);
    add_variants<255, 128, 3, 8, 1>(v);
    add_variants<255, 128, 2, 8, 1>(v);
    add_variants<255, 64, 4, 8, 1>(v);
    add_variants<255, 64, 2, 16, 1>(v);
}

}  // namespace hd
