"""Writes m2l_gen.cuh: straight-line float32 code for the mutual M2L at fixed order P.

For each P in 1..6 it emits
  m2l_dtensor_P(dx, dy, dz, soft2, D)   derivative tensor D^k(d), |k| <= P, of G = -(|d|^2 + soft2)^(-1/2)
                                         by the auxiliary recurrence R^(m)_{k+e_a} = d_a R^(m+1)_k + k_a R^(m+1)_{k-e_a}
  m2l_side_a_P(D, Ms, rho, L)           L^n = sum_j (-1)^|j| rho^|j| Ms^j D^{n+j}   (Ms = M/j!)
  m2l_side_b_P(D, Ms, L)                L^n = (-1)^|n| sum_j Ms^j D^{n+j}
(both overwrite L: the j = 0 term, which reaches every n, initialises it), and the variants
  m2l_side_a_forces_P, m2l_side_b_forces_P for accelerations only: L^0 (the potential term) is set to
  zero and the |j| = p moments, which only reach L^0, are not read.
Everything is unrolled with compile-time indices so that D and L live in registers.
Multi-indices are ordered by total degree, then nx descending, then ny descending.
Run: python gen_m2l.py > m2l_gen.cuh
"""

PMAX_GEN = 6


def multi_indices(p):
    mi = []
    for o in range(p + 1):
        for nx in range(o, -1, -1):
            for ny in range(o - nx, -1, -1):
                mi.append((nx, ny, o - nx - ny))
    return mi


def gen(P):
    mi = multi_indices(P)
    idx = {v: i for i, v in enumerate(mi)}
    nc = len(mi)
    out = []
    out.append(f"__device__ __forceinline__ void m2l_dtensor_{P}(float dx, float dy, float dz, float soft2, float (&D)[{nc}])")
    out.append("{")
    out.append("    const float s2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, soft2)));")
    out.append("    float si = rsqrtf(s2);")
    out.append("    si = si * fmaf(-0.5f * s2, si * si, 1.5f);   // one Newton step")
    out.append("    const float si2 = si * si;")
    out.append("    const float f0 = -si;")
    for m in range(1, P + 1):
        out.append(f"    const float f{m} = {-(2 * m - 1)}.0f * f{m - 1} * si2;")
    # R^(m)_k named r_m_k ; r_m_0 = f_m
    for m in range(P + 1):
        out.append(f"    const float r_{m}_0 = f{m};")
    axis_name = ["dx", "dy", "dz"]
    for k in range(1, nc):
        v = list(mi[k])
        a = 0 if v[0] > 0 else (1 if v[1] > 0 else 2)
        ka = v[a]
        w = list(v)
        w[a] -= 1
        km = idx[tuple(w)]
        kmm = None
        if ka >= 2:
            w2 = list(w)
            w2[a] -= 1
            kmm = idx[tuple(w2)]
        o = sum(v)
        for m in range(P - o + 1):
            expr = f"{axis_name[a]} * r_{m + 1}_{km}"
            if kmm is not None:
                expr = f"fmaf({float(ka - 1)}f, r_{m + 1}_{kmm}, {expr})"
            out.append(f"    const float r_{m}_{k} = {expr};")
    for k in range(nc):
        out.append(f"    D[{k}] = r_0_{k};")
    out.append("}")
    out.append("")
    for pot in (True, False):
        suf = "" if pot else "_forces"
        first_n = 0 if pot else 1   # forces only: L^0 (the potential term) is left at zero
        # side A: L^n = sum_j (-1)^|j| rho^|j| Ms^j D^{n+j}
        out.append(f"__device__ __forceinline__ void m2l_side_a{suf}_{P}(const float (&D)[{nc}], const float *__restrict__ Ms, float rho, float (&L)[{nc}])")
        out.append("{")
        if not pot:
            out.append("    L[0] = 0.0f;")
        out.append("    float rp = 1.0f;")
        prev_order = 0
        for j, (jx, jy, jz) in enumerate(mi):
            oj = jx + jy + jz
            if not pot and oj == P:
                continue   # only reaches n = 0
            if oj != prev_order:
                out.append("    rp *= rho;")
                prev_order = oj
            neg = (oj % 2) == 1
            out.append(f"    {{ const float m = {'-' if neg else ''}__ldg(Ms + {j}) * rp;")
            for n, (nx, ny, nz) in enumerate(mi):
                if n < first_n or nx + ny + nz + oj > P:
                    continue
                t = idx[(nx + jx, ny + jy, nz + jz)]
                if j == 0:
                    out.append(f"      L[{n}] = D[{t}] * m;")
                else:
                    out.append(f"      L[{n}] = fmaf(D[{t}], m, L[{n}]);")
            out.append("    }")
        out.append("}")
        out.append("")
        # side B: L^n = (-1)^|n| sum_j Ms^j D^{n+j}
        out.append(f"__device__ __forceinline__ void m2l_side_b{suf}_{P}(const float (&D)[{nc}], const float *__restrict__ Ms, float (&L)[{nc}])")
        out.append("{")
        if not pot:
            out.append("    L[0] = 0.0f;")
        for j, (jx, jy, jz) in enumerate(mi):
            oj = jx + jy + jz
            if not pot and oj == P:
                continue
            out.append(f"    {{ const float m = __ldg(Ms + {j});")
            for n, (nx, ny, nz) in enumerate(mi):
                on = nx + ny + nz
                if n < first_n or on + oj > P:
                    continue
                t = idx[(nx + jx, ny + jy, nz + jz)]
                sign = "-" if on % 2 else ""
                if j == 0:
                    out.append(f"      L[{n}] = {sign}D[{t}] * m;")
                else:
                    out.append(f"      L[{n}] = fmaf({sign}D[{t}], m, L[{n}]);")
            out.append("    }")
        out.append("}")
        out.append("")
    return "\n".join(out)


def main():
    print("// Generated by gen_m2l.py -- fixed-order float32 M2L building blocks (do not edit).")
    print("#pragma once")
    print()
    for P in range(1, PMAX_GEN + 1):
        print(gen(P))
    print("template <int P> struct M2LGen;")
    for P in range(1, PMAX_GEN + 1):
        nc = len(multi_indices(P))
        print(f"template <> struct M2LGen<{P}> {{")
        print(f"    static constexpr int NC = {nc};")
        print(f"    static __device__ __forceinline__ void dtensor(float dx, float dy, float dz, float s, float (&D)[{nc}]) {{ m2l_dtensor_{P}(dx, dy, dz, s, D); }}")
        print(f"    static __device__ __forceinline__ void side_a(const float (&D)[{nc}], const float *Ms, float rho, float (&L)[{nc}]) {{ m2l_side_a_{P}(D, Ms, rho, L); }}")
        print(f"    static __device__ __forceinline__ void side_b(const float (&D)[{nc}], const float *Ms, float (&L)[{nc}]) {{ m2l_side_b_{P}(D, Ms, L); }}")
        print(f"    static __device__ __forceinline__ void side_a_forces(const float (&D)[{nc}], const float *Ms, float rho, float (&L)[{nc}]) {{ m2l_side_a_forces_{P}(D, Ms, rho, L); }}")
        print(f"    static __device__ __forceinline__ void side_b_forces(const float (&D)[{nc}], const float *Ms, float (&L)[{nc}]) {{ m2l_side_b_forces_{P}(D, Ms, L); }}")
        print("};")


if __name__ == "__main__":
    main()
