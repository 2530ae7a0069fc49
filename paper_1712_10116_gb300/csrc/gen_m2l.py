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

For G = -1/|d| (no softening in the expansion) D^k is harmonic: D^{k+2e_x} + D^{k+2e_y} + D^{k+2e_z} = 0.
The harmonic set (m2l_*_h_P, M2LGenH<P>) uses it twice, without changing any result in exact arithmetic:
  * a moment component with j_z >= 2 meets D^{n+j} = -D^{n+j-2e_z+2e_x} - D^{n+j-2e_z+2e_y}, so it can be
    moved onto those two lower components once per cell (m2l_reduce_moments_h_P, highest j_z first);
    only the (p+1)^2 components with j_z <= 1 are then contracted;
  * the local coefficients inherit the relation, L^{n+2e_z} = -L^{n+2e_x} - L^{n+2e_y} (all three sums
    run over the same j), so only those with n_z <= 1 are formed per pair and the rest is filled in
    once per cell (m2l_complete_locals_h_P);
  * D is needed for k_z <= 2 only: the recurrence runs over (k_x, k_y) with k_z = 0, the k_z = 1
    components take one step along z, and the k_z = 2 ones follow from the harmonic relation.
For the directed form (one target cell, its sources one after another) m2l_acc_h[_forces]_P adds one
source's contribution to the target's reduced locals: L^n += sum_j (-1)^|j| rho^|j| Mr^j D^{n+j}.
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


def gen_h(P):
    """The harmonic set of order P (see the module docstring)."""
    mi = multi_indices(P)
    idx = {v: i for i, v in enumerate(mi)}
    nc = len(mi)
    H = [k for k in mi if k[2] <= 1]        # reduced moments and locals
    hidx = {v: i for i, v in enumerate(H)}
    DS = [k for k in mi if k[2] <= 2]       # derivative components the contractions read
    didx = {v: i for i, v in enumerate(DS)}
    nh, nd = len(H), len(DS)
    out = []
    out.append(f"__device__ __forceinline__ void m2l_dtensor_h_{P}(float dx, float dy, float dz, float (&D)[{nd}])")
    out.append("{")
    out.append("    const float s2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));")
    out.append("    float si = rsqrtf(s2);")
    out.append("    si = si * fmaf(-0.5f * s2, si * si, 1.5f);   // one Newton step")
    out.append("    const float si2 = si * si;")
    out.append("    const float f0 = -si;")
    for m in range(1, P + 1):
        out.append(f"    const float f{m} = {-(2 * m - 1)}.0f * f{m - 1} * si2;")
    for m in range(P + 1):
        out.append(f"    const float r_{m}_0 = f{m};")
    axis_name = ["dx", "dy", "dz"]
    # k_z = 0: the recurrence along x and y at every auxiliary level it feeds
    for k in range(1, nc):
        v = list(mi[k])
        if v[2] != 0:
            continue
        a = 0 if v[0] > 0 else 1
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
    for k, v in enumerate(DS):
        if v[2] == 0:
            out.append(f"    D[{k}] = r_0_{idx[v]};")
        elif v[2] == 1:
            # R^(0)_{k'+e_z} = d_z R^(1)_{k'} (k'_z = 0, so the second term vanishes)
            out.append(f"    D[{k}] = dz * r_1_{idx[(v[0], v[1], 0)]};")
    for k, v in enumerate(DS):
        if v[2] == 2:
            out.append(f"    D[{k}] = -D[{didx[(v[0] + 2, v[1], 0)]}] - D[{didx[(v[0], v[1] + 2, 0)]}];")
    out.append("}")
    out.append("")
    for pot in (True, False):
        suf = "" if pot else "_forces"
        first_n = 0 if pot else 1
        out.append(f"__device__ __forceinline__ void m2l_side_a_h{suf}_{P}(const float (&D)[{nd}], const float *__restrict__ Mr, float rho, float (&L)[{nh}])")
        out.append("{")
        if not pot:
            out.append("    L[0] = 0.0f;")
        out.append("    float rp = 1.0f;")
        prev_order = 0
        for j, (jx, jy, jz) in enumerate(H):
            oj = jx + jy + jz
            if not pot and oj == P:
                continue
            if oj != prev_order:
                out.append("    rp *= rho;")
                prev_order = oj
            neg = (oj % 2) == 1
            out.append(f"    {{ const float m = {'-' if neg else ''}__ldg(Mr + {j}) * rp;")
            for n, (nx, ny, nz) in enumerate(H):
                if n < first_n or nx + ny + nz + oj > P:
                    continue
                t = didx[(nx + jx, ny + jy, nz + jz)]
                if j == 0:
                    out.append(f"      L[{n}] = D[{t}] * m;")
                else:
                    out.append(f"      L[{n}] = fmaf(D[{t}], m, L[{n}]);")
            out.append("    }")
        out.append("}")
        out.append("")
        # directed accumulation: L^n += sum_j (-1)^|j| rho^|j| Mr^j D^{n+j} (one target, one source)
        out.append(f"__device__ __forceinline__ void m2l_acc_h{suf}_{P}(const float (&D)[{nd}], const float *__restrict__ Mr, float rho, float (&L)[{nh}])")
        out.append("{")
        out.append("    float rp = 1.0f;")
        prev_order = 0
        for j, (jx, jy, jz) in enumerate(H):
            oj = jx + jy + jz
            if not pot and oj == P:
                continue
            if oj != prev_order:
                out.append("    rp *= rho;")
                prev_order = oj
            neg = (oj % 2) == 1
            out.append(f"    {{ const float m = {'-' if neg else ''}__ldg(Mr + {j}) * rp;")
            for n, (nx, ny, nz) in enumerate(H):
                if n < first_n or nx + ny + nz + oj > P:
                    continue
                t = didx[(nx + jx, ny + jy, nz + jz)]
                out.append(f"      L[{n}] = fmaf(D[{t}], m, L[{n}]);")
            out.append("    }")
        out.append("}")
        out.append("")
        out.append(f"__device__ __forceinline__ void m2l_side_b_h{suf}_{P}(const float (&D)[{nd}], const float *__restrict__ Mr, float (&L)[{nh}])")
        out.append("{")
        if not pot:
            out.append("    L[0] = 0.0f;")
        for j, (jx, jy, jz) in enumerate(H):
            oj = jx + jy + jz
            if not pot and oj == P:
                continue
            out.append(f"    {{ const float m = __ldg(Mr + {j});")
            for n, (nx, ny, nz) in enumerate(H):
                on = nx + ny + nz
                if n < first_n or on + oj > P:
                    continue
                t = didx[(nx + jx, ny + jy, nz + jz)]
                sign = "-" if on % 2 else ""
                if j == 0:
                    out.append(f"      L[{n}] = {sign}D[{t}] * m;")
                else:
                    out.append(f"      L[{n}] = fmaf({sign}D[{t}], m, L[{n}]);")
            out.append("    }")
        out.append("}")
        out.append("")
    # per cell: fold the j_z >= 2 moments down (highest j_z first), keep the j_z <= 1 ones
    out.append(f"__device__ __forceinline__ void m2l_reduce_moments_h_{P}(const float *__restrict__ Ms, float *__restrict__ Mr)")
    out.append("{")
    for k in range(nc):
        out.append(f"    float v{k} = Ms[{k}];")
    for jz in range(P, 1, -1):
        for k, v in enumerate(mi):
            if v[2] != jz:
                continue
            ax = idx[(v[0] + 2, v[1], v[2] - 2)]
            ay = idx[(v[0], v[1] + 2, v[2] - 2)]
            out.append(f"    v{ax} -= v{k};")
            out.append(f"    v{ay} -= v{k};")
    for h, v in enumerate(H):
        out.append(f"    Mr[{h}] = v{idx[v]};")
    out.append("}")
    out.append("")
    # per cell: the locals with n_z >= 2 from the harmonic relation (their two partners come earlier)
    out.append(f"__device__ __forceinline__ void m2l_complete_locals_h_{P}(const float *__restrict__ Lr, float *__restrict__ L)")
    out.append("{")
    for k, v in enumerate(mi):
        if v[2] <= 1:
            out.append(f"    const float v{k} = Lr[{hidx[v]}];")
        else:
            out.append(f"    const float v{k} = -v{idx[(v[0] + 2, v[1], v[2] - 2)]} - v{idx[(v[0], v[1] + 2, v[2] - 2)]};")
        out.append(f"    L[{k}] = v{k};")
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
    for P in range(1, PMAX_GEN + 1):
        print(gen_h(P))
    print("template <int P> struct M2LGenH;")
    for P in range(1, PMAX_GEN + 1):
        mi = multi_indices(P)
        nh = sum(1 for k in mi if k[2] <= 1)
        nd = sum(1 for k in mi if k[2] <= 2)
        print(f"template <> struct M2LGenH<{P}> {{")
        print(f"    static constexpr int NC = {nh};")
        print(f"    static constexpr int ND = {nd};")
        print(f"    static __device__ __forceinline__ void dtensor(float dx, float dy, float dz, float (&D)[{nd}]) {{ m2l_dtensor_h_{P}(dx, dy, dz, D); }}")
        print(f"    static __device__ __forceinline__ void side_a(const float (&D)[{nd}], const float *Mr, float rho, float (&L)[{nh}]) {{ m2l_side_a_h_{P}(D, Mr, rho, L); }}")
        print(f"    static __device__ __forceinline__ void side_b(const float (&D)[{nd}], const float *Mr, float (&L)[{nh}]) {{ m2l_side_b_h_{P}(D, Mr, L); }}")
        print(f"    static __device__ __forceinline__ void side_a_forces(const float (&D)[{nd}], const float *Mr, float rho, float (&L)[{nh}]) {{ m2l_side_a_h_forces_{P}(D, Mr, rho, L); }}")
        print(f"    static __device__ __forceinline__ void side_b_forces(const float (&D)[{nd}], const float *Mr, float (&L)[{nh}]) {{ m2l_side_b_h_forces_{P}(D, Mr, L); }}")
        print(f"    static __device__ __forceinline__ void acc(const float (&D)[{nd}], const float *Mr, float rho, float (&L)[{nh}]) {{ m2l_acc_h_{P}(D, Mr, rho, L); }}")
        print(f"    static __device__ __forceinline__ void acc_forces(const float (&D)[{nd}], const float *Mr, float rho, float (&L)[{nh}]) {{ m2l_acc_h_forces_{P}(D, Mr, rho, L); }}")
        print(f"    static __device__ __forceinline__ void reduce_moments(const float *Ms, float *Mr) {{ m2l_reduce_moments_h_{P}(Ms, Mr); }}")
        print(f"    static __device__ __forceinline__ void complete_locals(const float *Lr, float *L) {{ m2l_complete_locals_h_{P}(Lr, L); }}")
        print("};")


if __name__ == "__main__":
    main()
