"""Write fcs_roots.cuh: cos and sin of 2 pi k / N for the small DFT sizes of
the register FFT, to 20 significant digits (mpmath), as constant-memory
tables.  Run: python gen_roots.py > fcs_roots.cuh"""
import mpmath as mp

SIZES = (2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 14, 16, 18, 20, 24, 28, 32, 36, 40)
mp.mp.dps = 30


def main():
    offs, vals = {}, []
    for N in SIZES:
        offs[N] = len(vals)
        for k in range(N):
            a = -2 * mp.pi * k / N          # forward roots e^{-2 pi i k / N}
            vals.append((mp.cos(a), mp.sin(a)))
    print("// Generated by gen_roots.py: e^{-2 pi i k / N} for the register-DFT sizes.")
    print("#pragma once")
    print("namespace fcs {")
    print("__host__ __device__ constexpr int kRootOff(int N) {")
    print("  return " + " : ".join(f"N == {N} ? {offs[N]}" for N in SIZES) + " : -1;")
    print("}")
    for ty, name, suffix in (("double2", "kRoots64", ""), ("float2", "kRoots32", "f")):
        print(f"static __constant__ {ty} {name}[{len(vals)}] = {{")
        for c, s in vals:
            print(f"    {{{mp.nstr(c, 20, min_fixed=-1, max_fixed=1)}{suffix}, {mp.nstr(s, 20, min_fixed=-1, max_fixed=1)}{suffix}}},")
        print("};")
    print("}  // namespace fcs")


if __name__ == "__main__":
    main()
