// hd_multi_a.cu -- compiled multi-packet streaming configurations for n = 7,
// 15 and 31: the single-stream decoder's built-in chunk geometry per n (n = 7
// and 15 with their decode tables, and without them for a first plan launch
// that is captured before the tables exist).
#include "hd_multi.cuh"

namespace hd {

void register_multi_a(std::vector<MultiVariant> &v)
{
    add_multi_variants<7, 128, 4, 32, 1, true>(v);
    add_multi_variants<7, 128, 4, 32, 1>(v);
    add_multi_variants<15, 576, 2, 32, 0, true>(v);
    add_multi_variants<15, 256, 4, 32, 1>(v);
    add_multi_variants<31, 128, 2, 32, 1>(v);
}

}  // namespace hd
