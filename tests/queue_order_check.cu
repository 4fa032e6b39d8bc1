// queue_order_check.cu -- host program that checks the work-queue orders of
// the persistent kernels with their own decoders (decode_item in persist.cuh,
// three_decode in threestep.cuh), compiled for the host; no GPU is used.
//
// For each parameter set on the command line it enumerates every queue
// position and checks
//   * the decoder is a bijection onto the tiles (each tile exactly once);
//   * every tile that waits is preceded in the queue by all the tiles it
//     waits for (two-pass: a second-pass tile of chunk j after all na
//     first-pass tiles of chunk j; three-stage: a B1 tile of chunk c after
//     all na A tiles of chunk c, a B2 tile of group (c, g) after all nb1g B1
//     tiles of (c, g)).
// Together with "a CTA holds one item at a time and publishes its signal
// before it waits", this is why every bounded wait of those kernels ends.
// It prints the smallest distance in queue positions between a waiting tile
// and the last tile it needs, per kind, and exits non-zero on a violation.
//
//   queue_order_check [--plant] two  na nb nch
//   queue_order_check [--plant] three na nch G nb1g nb2g D
// --plant attributes every decoded second-pass (B1) tile to the chunk two
// ahead (a decoder that runs the second pass early), to show that the check
// sees it.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../paper_1203_4938_b300/csrc/threestep.cuh"

using b300fft::decode_item;
using b300fft::three_decode;

static bool g_plant = false;

static int fail(const char* what, long long p) {
    std::printf("FAIL %s at position %lld\n", what, p);
    return 1;
}

static int check_two(int na, int nb, int nch) {
    const long long total = (long long)nch * (na + nb);
    std::vector<long long> pos_a((size_t)nch * na, -1), pos_b((size_t)nch * nb, -1);
    for (long long p = 0; p < total; ++p) {
        bool is_b;
        int j, r;
        decode_item((int)p, na, nb, nch, &is_b, &j, &r);
        if (g_plant && is_b) j = (j + 2) % nch;
        if (j < 0 || j >= nch || r < 0 || r >= (is_b ? nb : na)) return fail("decoded tile out of range", p);
        long long& slot = is_b ? pos_b[(size_t)j * nb + r] : pos_a[(size_t)j * na + r];
        if (slot >= 0) return fail("tile decoded twice", p);
        slot = p;
    }
    long long lag = total;
    for (int j = 0; j < nch; ++j) {
        long long last_a = -1;
        for (int r = 0; r < na; ++r) last_a = pos_a[(size_t)j * na + r] > last_a ? pos_a[(size_t)j * na + r] : last_a;
        for (int r = 0; r < nb; ++r) {
            const long long pb = pos_b[(size_t)j * nb + r];
            if (pb <= last_a) return fail("second-pass tile before a first-pass tile it needs", pb);
            lag = pb - last_a < lag ? pb - last_a : lag;
        }
    }
    std::printf("OK two na=%d nb=%d nch=%d items=%lld min_lag=%lld\n", na, nb, nch, total, lag);
    return 0;
}

static int check_three(int na, int nch, int G, int nb1g, int nb2g, int D) {
    b300fft::ThreeArgs a{};
    a.na = na;
    a.nch = nch;
    a.G = G;
    a.nb1g = nb1g;
    a.nb2g = nb2g;
    a.D = D;
    a.nb = G * (nb1g + nb2g);
    const long long total = (long long)nch * (a.na + a.nb);
    std::vector<long long> pa((size_t)nch * na, -1), pb1((size_t)nch * G * nb1g, -1), pb2((size_t)nch * G * nb2g, -1);
    for (long long p = 0; p < total; ++p) {
        int st, c, g, r;
        three_decode(a, (int)p, &st, &c, &g, &r);
        if (g_plant && st == b300fft::kStageB1) c = (c + 2) % nch;
        if (c < 0 || c >= nch) return fail("chunk out of range", p);
        long long* slot = nullptr;
        if (st == b300fft::kStageA) {
            if (g != 0 || r < 0 || r >= na) return fail("A tile out of range", p);
            slot = &pa[(size_t)c * na + r];
        } else if (st == b300fft::kStageB1) {
            if (g < 0 || g >= G || r < 0 || r >= nb1g) return fail("B1 tile out of range", p);
            slot = &pb1[((size_t)c * G + g) * nb1g + r];
        } else if (st == b300fft::kStageB2) {
            if (g < 0 || g >= G || r < 0 || r >= nb2g) return fail("B2 tile out of range", p);
            slot = &pb2[((size_t)c * G + g) * nb2g + r];
        } else {
            return fail("unknown stage", p);
        }
        if (*slot >= 0) return fail("tile decoded twice", p);
        *slot = p;
    }
    long long lag1 = total, lag2 = total;
    for (int c = 0; c < nch; ++c) {
        long long last_a = -1;
        for (int r = 0; r < na; ++r) last_a = pa[(size_t)c * na + r] > last_a ? pa[(size_t)c * na + r] : last_a;
        for (int g = 0; g < G; ++g) {
            long long last_b1 = -1;
            for (int r = 0; r < nb1g; ++r) {
                const long long q = pb1[((size_t)c * G + g) * nb1g + r];
                if (q <= last_a) return fail("B1 tile before an A tile it needs", q);
                lag1 = q - last_a < lag1 ? q - last_a : lag1;
                last_b1 = q > last_b1 ? q : last_b1;
            }
            for (int r = 0; r < nb2g; ++r) {
                const long long q = pb2[((size_t)c * G + g) * nb2g + r];
                if (q <= last_b1) return fail("B2 tile before a B1 tile it needs", q);
                lag2 = q - last_b1 < lag2 ? q - last_b1 : lag2;
            }
        }
    }
    std::printf("OK three na=%d nch=%d G=%d nb1g=%d nb2g=%d D=%d items=%lld min_lag_b1=%lld min_lag_b2=%lld\n", na,
                nch, G, nb1g, nb2g, D, total, lag1, lag2);
    return 0;
}

int main(int argc, char** argv) {
    int bad = 0;
    int i = 1;
    if (i < argc && argv[i][0] == '-' && argv[i][1] == '-') {
        g_plant = true;
        ++i;
    }
    while (i < argc) {
        const char* kind = argv[i];
        if (kind[0] == 't' && kind[1] == 'w' && i + 3 < argc) {
            bad |= check_two(std::atoi(argv[i + 1]), std::atoi(argv[i + 2]), std::atoi(argv[i + 3]));
            i += 4;
        } else if (kind[0] == 't' && kind[1] == 'h' && i + 6 < argc) {
            bad |= check_three(std::atoi(argv[i + 1]), std::atoi(argv[i + 2]), std::atoi(argv[i + 3]),
                               std::atoi(argv[i + 4]), std::atoi(argv[i + 5]), std::atoi(argv[i + 6]));
            i += 7;
        } else {
            std::printf("usage: %s [--plant] two na nb nch | three na nch G nb1g nb2g D ...\n", argv[0]);
            return 2;
        }
    }
    return bad;
}
