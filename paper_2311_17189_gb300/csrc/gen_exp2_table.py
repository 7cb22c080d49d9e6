"""Writes the two-part table of 2^(j/256), j = 0..255, that the kernels' exponential reads
(tami_devmath.cuh, kExp2TabHi / kExp2TabLo): T_hi is 2^(j/256) rounded to the nearest double and
T_lo the nearest double to the remainder, both from 60-digit values.  Run it to regenerate the
arrays (printed as C); tests/test_devmath_tables_cpu.py checks the header against it."""
import mpmath as mp

N = 256


def table():
    mp.mp.dps = 60
    hi, lo = [], []
    for j in range(N):
        v = mp.power(2, mp.mpf(j) / N)
        h = float(v)
        hi.append(h)
        lo.append(float(v - mp.mpf(h)))
    return hi, lo


def c_arrays():
    hi, lo = table()

    def block(name, vals):
        lines = []
        for i in range(0, N, 4):
            lines.append("  " + ", ".join(v.hex() if v != 0.0 else "0x0.0p+0" for v in vals[i:i + 4]))
        return "__device__ const double %s[%d] = {\n%s};" % (name, N, ",\n".join(lines))

    return block("kExp2TabHi", hi) + "\n" + block("kExp2TabLo", lo)


if __name__ == "__main__":
    print(c_arrays())
