// hd_stream_x.cu -- the SECDED configurations of the streaming decoder, one
// per length n (codewords per thread, threads per CTA, stages, in-place), for
// every syndrome type: the fastest of a sweep of configurations on GB300; for
// n = 7 and 15 also one with the SECDED decode table.
#include "hd_stream.cuh"

namespace hd {

void register_stream_secded(std::vector<StreamVariant> &v)
{
    // the first arithmetic configuration of each n is its default: the fastest
    // of a sweep over rotating buffer sets at 2^24 (n <= 63) or 2^22 codewords
    // on GB300 (n = 127: 26.5 µs against 29.0 for 128 threads, 2 stages, G = 8)
    add_variants<7, 128, 4, 32, 1, true>(v);
    add_variants<15, 512, 2, 32, 1, true>(v);
    add_variants<31, 256, 2, 32, 1, true>(v);
    add_variants<63, 64, 2, 32, 1, true>(v);
    add_variants<127, 64, 3, 16, 1, true>(v);
    add_variants<255, 128, 2, 8, 1, true>(v);
    // decode tables (one lookup per codeword; used when the table is filled)
    add_variants<7, 128, 4, 32, 1, true, true>(v);
    add_variants<15, 512, 2, 32, 1, true, true>(v);  // 128 KB table per CTA
    // further configurations, selectable with hd_secded_variant_select
    add_variants<31, 128, 4, 32, 1, true>(v);
    add_variants<31, 128, 2, 32, 1, true>(v);
    add_variants<63, 128, 2, 32, 1, true>(v);
    add_variants<63, 128, 3, 32, 1, true>(v);
    add_variants<127, 128, 2, 8, 1, true>(v);
    add_variants<127, 256, 3, 8, 1, true>(v);
    add_variants<127, 128, 2, 16, 1, true>(v);
    add_variants<255, 128, 3, 8, 1, true>(v);
    add_variants<255, 64, 2, 16, 1, true>(v);
    add_variants<15, 384, 2, 32, 1, true, true>(v);
}

}  // namespace hd
