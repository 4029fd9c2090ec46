"""The benchmark's clock record on the CPU: the nvidia-smi samples taken during
the timed region are reduced to the median SM clock under load, the maximum
clock and the active throttle reasons (a run with a thermal or hardware
slowdown is one to reject)."""
import bench


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def record(rows):
    c = bench.Clocks(0)
    c.f.write("".join(r + "\n" for r in rows))
    c.p = _Done()
    return c.stop()


NOT = "Not Active"


def row(sm, mx=2070, hw=NOT, hwt=NOT, swt=NOT, swp=NOT):
    return "0, %d, %d, 900.00, 0x0000000000000000, %s, %s, %s, %s" % (sm, mx, hw, hwt, swt, swp)


def test_median_under_load_and_no_reasons():
    r = record([row(345), row(2070), row(2070), row(2055), row(2070)])
    assert r["sm_max_mhz"] == 2070 and r["reasons"] == [] and r["samples"] == 5
    assert r["sm_mhz"] == 2070  # the idle sample below half the maximum is left out


def test_throttle_reasons_are_reported():
    r = record([row(2070), row(1800, hwt="Active"), row(1900, swp="Active")])
    assert r["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    r = record([row(2070, hw="Active"), row(2070, swt="Active")])
    assert r["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_no_samples():
    assert record([]) is None
    assert record(["garbage line"]) is None
