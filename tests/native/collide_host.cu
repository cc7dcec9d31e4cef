// Host-side harness: runs the library's fused collision (compiled for the CPU
// from the same device header) on node states read from stdin, so that its
// arithmetic can be checked against the FP64 oracle without a GPU.
//
// stdin:  s_e s_q q_k q_e a_T gbeta bf0 bf1 bf2, then lines of 26 values
//         (19 f deviations f - w rho0, 7 g)
// stdout: per node 26 post-collision values, then rho-1 u v w T
// argv[1] == "double": the same collision instantiated in FP64 (the rates and
// the constants of the collision stay FP32 numbers), which separates the
// algebra from the FP32 rounding.
#include <cstdio>
#include <cstring>

#include "../../paper_1903_08882_gb300/csrc/lbm_device.cuh"

template <typename V> int run(const lbm::Phys &P) {
    V f[19], g[7];
    for (;;) {
        double x;
        for (int i = 0; i < 19; ++i) {
            if (std::scanf("%lf", &x) != 1) return 0;
            f[i] = (V)x;
        }
        for (int i = 0; i < 7; ++i) {
            if (std::scanf("%lf", &x) != 1) return 1;
            g[i] = (V)x;
        }
        const lbm::MacroT<V> m = lbm::collide(P, f, g);
        for (int i = 0; i < 19; ++i) std::printf("%.17e ", (double)f[i]);
        for (int i = 0; i < 7; ++i) std::printf("%.17e ", (double)g[i]);
        std::printf("%.17e %.17e %.17e %.17e %.17e\n", (double)m.drho, (double)m.u, (double)m.v, (double)m.w,
                    (double)m.T);
    }
}

int main(int argc, char **argv) {
    lbm::Phys P{};
    if (std::scanf("%f %f %f %f %f %f %f %f %f", &P.s_e, &P.s_q, &P.q_k, &P.q_e, &P.a_T, &P.gbeta, &P.bf[0],
                   &P.bf[1], &P.bf[2]) != 9)
        return 1;
    if (argc > 1 && std::strcmp(argv[1], "double") == 0) return run<double>(P);
    return run<float>(P);
}
