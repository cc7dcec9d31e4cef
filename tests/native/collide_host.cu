// Host-side harness: runs the library's fused collision (compiled for the CPU
// from the same device header) on node states read from stdin, so that its
// arithmetic can be checked against the FP64 oracle without a GPU.
//
// stdin:  s_e s_q q_k q_e a_T gbeta bf0 bf1 bf2, then lines of 26 floats
//         (19 f deviations f - w rho0, 7 g)
// stdout: per node 26 post-collision values, then rho-1 u v w T
#include <cstdio>

#include "../../paper_1903_08882_gb300/csrc/lbm_device.cuh"

int main() {
    lbm::Phys P{};
    if (std::scanf("%f %f %f %f %f %f %f %f %f", &P.s_e, &P.s_q, &P.q_k, &P.q_e, &P.a_T, &P.gbeta, &P.bf[0],
                   &P.bf[1], &P.bf[2]) != 9)
        return 1;
    float f[19], g[7];
    for (;;) {
        for (int i = 0; i < 19; ++i)
            if (std::scanf("%f", &f[i]) != 1) return 0;
        for (int i = 0; i < 7; ++i)
            if (std::scanf("%f", &g[i]) != 1) return 1;
        const lbm::Macro m = lbm::collide(P, f, g);
        for (int i = 0; i < 19; ++i) std::printf("%.9e ", f[i]);
        for (int i = 0; i < 7; ++i) std::printf("%.9e ", g[i]);
        std::printf("%.9e %.9e %.9e %.9e %.9e\n", m.drho, m.u, m.v, m.w, m.T);
    }
}
